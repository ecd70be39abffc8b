"""Plain FP64 CPU oracle for the 2-D Lippmann-Schwinger Nystrom operator.

TEST INFRASTRUCTURE ONLY.  Nothing in the library (``paper_1509_05063_gb300``)
imports, links or executes anything here; only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use it.
It shares no code with the CUDA path: geometry, quadrature, interpolation,
singular rules, the direct O(N^2) operator, the equivalent-source accelerator,
GMRES, the series solutions and the far field are all written out here from the
paper (arXiv:1509.05063) with numpy / scipy as the only helpers.

Modules
-------
geometry    charts, partition of unity, Nystrom nodes and weights   (Sec. 2, Sec. 3)
quadrature  cut-off, Newton-Cotes, Lagrange interpolation, singular rules (Sec. 3.1)
operator    direct apply u + kappa^2 K[u] with exact far sum (Eq. VolInt-Adj-NonAdj-I)
accel       equivalent-source / lattice-FFT / local-expansion accelerator (Sec. 3.2)
gmres       restarted GMRES in complex FP64 (Sec. 2)
exact       Bessel-series disc solution, closed-form volume potential, far field
"""
