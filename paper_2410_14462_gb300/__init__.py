"""libludvig: GB300-native feature uplifting onto 3D Gaussian Splatting scenes.

The compute path lives in the CUDA shared library ``libludvig.so`` (built from
``csrc/``); :mod:`paper_2410_14462_gb300.ludvig` is its thin ctypes binding and
:mod:`paper_2410_14462_gb300.inputs` holds the seeded synthetic workload
generators.  Nothing is imported eagerly so that the generators can be used on
a machine without the CUDA library.
"""
