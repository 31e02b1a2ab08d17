"""GB300-native (sm_103a) implementation of the HOBI-PB boundary integral solver.

* ``hobi``  -- ctypes binding of ``libhobi.so`` (the C ABI in ``include/hobi.h``)
* ``synth`` -- seeded synthetic inputs (icospheres, charges, molecular surfaces)
* ``build`` -- nvcc build of the CUDA library
"""
