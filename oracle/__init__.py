"""FP64 CPU oracle for the parallel square-root smoothers of arXiv 2207.00426.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.  It shares no code with the CUDA path.

It is deliberately plain and slow: NumPy in float64, sequential loops over
time steps, library primitives (QR, Cholesky, solves) used as single steps.
Every function names the section, table, lemma, algorithm or equation of the
paper that it follows.

Modules
-------
linalg    Tria (Sec. 2.2) and DownDate (Sec. 2.2).
kalman    Sequential square-root and covariance Kalman filter / RTS smoother
          and the per-step log-likelihood (Sec. 5.1).
parallel  Square-root and standard scan elements and operators
          (Lemmas 1-4, Tables 1-5) and scan orders (Alg. 1, Alg. 2).
models    Coordinated-turn bearings-only model and the linear
          constant-velocity model used by the experiments (Sec. 6).
slr       Taylor (Sec. 4.2) and cubature sigma-point (Sec. 4.3) square-root
          statistical linear regression.
ipls      Iterated posterior linearisation (Alg. 3), pseudo log-likelihood
          (Sec. 5.1) and its gradient by central finite differences (Sec. 5.2).
"""
