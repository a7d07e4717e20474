"""Plain CPU FP64 oracle for the Flux Reconstruction (FR) right-hand side.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library (``paper_2408_16509_gb300``) and never imports it.

What it computes (PyFR v2.0.3, arXiv 2408.16509, Section 2):

* Eq. (disu, first form): discontinuous solution at flux points,
  ``u_f = sum_z u_z l_z(x_f)``                                (``fr.interp``)
* Eq. (comm_flux): common normal flux at flux points from both sides'
  states and the surface normal -- a Rusanov Riemann solver (``physics``)
* Eq. (disu, second form): transformed discontinuous normal flux at the
  flux points ``n . sum_z f~_z l_z(x_f)``
* Eq. (FRfinal): corrected divergence
  ``sum_s div g_s (F^C_s - f_s) + sum_v f~_v . grad l_v``      (``fr.rhs``)
* Section 2 transformed equation: ``du/dt = -J^{-1} div~ f~``
* explicit Runge-Kutta time integration                       (``rk``)

Everything is FP64 numpy, dense operator matrices built from Vandermonde
matrices of orthonormal bases, per-element loops written as batched matrix
products over elements (a library matmul as one step), no fusion: the
interpolation, divergence and correction operators are applied separately.

Parity status per function is recorded in each module header; the pins that
tie it to the paper and to mathematics live in ``tests/test_oracle_*.py``.
"""
