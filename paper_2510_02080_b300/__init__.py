"""B300-native hot path of EC3R-SLAM submap fusion.

``ec3r`` is the ctypes binding of the C-ABI library ``libec3r.so`` (CUDA for
sm_103a): batched Huber-IRLS Umeyama Sim(3) registration, the Sim(3)
pose-graph Gauss-Newton correction, confidence-filtered fusion and the
adjoint of the registration.  ``synth`` generates seeded synthetic inputs.
Importing this package loads nothing; ``ec3r.lib()`` loads the library.
"""
