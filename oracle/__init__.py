"""Plain FP64 CPU oracle for the JFNK-GMRES / DG->FV multigrid hot path.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py may import or run anything here.
The CUDA library never imports, links or calls it, and it shares no code,
tables or constants with the CUDA path: every table is recomputed here
with numpy.

It follows Birken, Dedner, Kloefkorn, "A Jacobian-free multigrid
preconditioner for DG methods applied to NWP" (arXiv 2505.24504):
  tables.py  Gauss-Legendre nodal Q_k basis (Sec. 2.1), FV subcell centres,
             interpolation transfer and the modified Newton-Cotes weights
             (Sec. 3.2.2, Appendix A).
  physics.py Euler/viscous model with gravity, EOS, environmental atmospheres,
             pressure-preserving perturbation insertion, HLLC (Sec. 4, eq.
             compressible-euler, eq. add-perturbation).
  dg.py      well-balanced DG operator f = M^-1 L_h (eqs. convDiscr,
             elementint, surfaceint, perturbed-euler) and the FD Jacobian-
             vector product (Sec. 3.1).
  fv.py      FV subgrid operator f_low, agglomeration hierarchy, R, P,
             pseudo-time smoother, MG V/W cycle, transfer with mass fix
             (Sec. 3.2-3.5).
  solver.py  FGMRES, Eisenstat-Walker Newton, SDIRK2 / backward Euler
             (Sec. 2.2, 3.1).

Every function works on float64 arrays; the DG operator also accepts
complex128 input (comparisons use real parts) so that complex-step
derivatives give an exact Jacobian for pinning the FD product.

Parity unpinned: the pseudo-time step sizes of the smoothers (sigma,
lambda), the interior-penalty constant C_IP and the DG pre/post
smoothing order affect iteration counts only; no value in the paper
fixes them.
"""
