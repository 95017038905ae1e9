"""FP64 CPU oracle of the EC3R-SLAM submap-fusion hot path.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute anything in this package: only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

It is a plain, slow, obviously-correct restatement of what the path computes,
in float64 numpy, written from the paper:

* ``sim3``        - Sim(3) group algebra, Exp/Log from their definitions
                    (matrix exponential of the 4x4 generator), used by the
                    pose graph (Sec. III-E).
* ``register``    - correspondence set-up, weighted Umeyama (Sec. III-C,
                    Eq. (sim3) and the weighted Umeyama solution) and the
                    Huber-IRLS loop around it.
* ``pose_graph``  - edge error e_ij = log(T_ij^-1 T_i^-1 T_j), chi^2,
                    chaining initialisation and Gauss-Newton (Sec. III-E).
* ``unproject``   - inverse projection of depth maps through pinhole cameras
                    (Sec. III-C "Feed-Forward Inference": submaps from the
                    predicted depths and cameras).
* ``fuse``        - confidence-filtered compaction and transform of submap
                    points into the global frame (Sec. III-C "Point
                    Correction": global coordinates of all submap points).
* ``adjoint``     - reverse-mode derivative of the IRLS registration.

It shares no code with the CUDA path (``paper_2510_02080_b300``); the only
common module is the seeded input generator ``paper_2510_02080_b300.synth``,
which contains no arithmetic of the method.  Every function is pinned by the
``-m "not gpu"`` tests in ``tests/test_oracle_*.py``.
"""
