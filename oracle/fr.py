"""The FR right-hand side, step by step (test infrastructure only).

Follows Section 2 of the paper in its order, element type by element type,
with dense operators and no fusion:

1. Eq. (disu): u_f = M0 u                                     (solution -> flux pts)
2. Eq. (comm_flux): F^C at every flux point from both sides (Rusanov; the
   boundary supplies the outside state).  Transformed normal common flux =
   |S^T n~| F^C(n) for the element's own outward normal.
3. transformed flux at solution points f~ = S f (S = det J J^{-1}), then
   Eq. (disu, second form): f~_n = n~ . (M0 f~)
4. Eq. (FRfinal): div = sum_d D_d f~_d + LIFT (F^C - f~_n)
5. du/dt = -div / det J   (the transformed equation of Section 2)

Navier-Stokes inserts the gradient path before step 3 (the paper names the
compressible NS solver but not its formulas; reading, BR1 of Bassi & Rebay):
common solution u^C = (u- + u+)/2, corrected reference gradient
grad~ u = D u + LIFT (n~ (u^C - u_f)), physical gradient (1/det J) S^T grad~ u,
gradient at flux points = M0 (physical gradient), viscous common flux =
average of both sides' viscous fluxes.  At a boundary flux point the outside
state comes from the boundary condition and the outside gradient equals the
inside one.

Anti-aliasing (Section 3.2, "Anti-aliasing"; ``antialias=qdeg``): step 3
takes the transformed flux at the points of a degree-qdeg volume rule
(u and, for NS, the physical gradient interpolated there, S evaluated
there) and replaces the collocated f~ by its least-squares projection onto
the solution space, f~ = P f~_q; steps 4 and 5 are unchanged.

LDG (``ldg=(beta, tau)``; the paper names no viscous scheme, reading of the
local DG flux of Cockburn and Shu): along every interface's orientation
(mesh.pair_l is the "-" side, a boundary's inside is "-" and its outside
state "+"), u^C = (1/2 - beta) u- + (1/2 + beta) u+, the viscous common
flux (1/2 + beta) F_v- + (1/2 - beta) F_v+ (biased the other way), and the
common normal flux gains the penalty tau (u- - u+).  beta = tau = 0 is BR1.

Boundary conditions (by tag): ('state', rho, u, v, w, p) -- outside state is
the given constant state; ('extrap',) -- outside state = inside state;
('prescribed', fn) -- outside state given point by point, fn(x) returning
the primitive state (rho, u, v, w, p) at the boundary flux points x (n, 3);
the outside gradient is the inside one in every case.
"""
import numpy as np

from .physics import euler_flux, prim_to_cons, rusanov, viscous_flux


class FRSystem:
    def __init__(self, mesh, physics="euler", gamma=1.4, mu=0.0, pr=0.72,
                 bcs=None, antialias=None, ldg=None):
        self.m = mesh
        self.beta, self.tau = (0.0, 0.0) if ldg is None else (float(ldg[0]), float(ldg[1]))
        self.aa = {}
        if antialias is not None:
            for t in mesh.types:
                xq, _, B, P = mesh.el[t].aa_operators(int(antialias))
                self.aa[t] = (B, P, mesh.metric_at(t, xq))
        self.physics = physics
        self.gamma, self.mu, self.pr = gamma, mu, pr
        self.bcs = dict(bcs or {})
        self._ghost_state = {}
        for tag, bc in self.bcs.items():
            if bc[0] == "state":
                rho, u, v, w, p = bc[1:]
                self._ghost_state[tag] = prim_to_cons(
                    np.array(rho), np.array([u, v, w]), np.array(p), gamma)

    # --- helpers -----------------------------------------------------------
    def interp(self, u):
        """Step 1, Eq. (disu): u at flux points, global flux-point order."""
        m = self.m
        return m.flat({t: np.einsum("fz,ezv->efv", m.el[t].M0, u[t])
                       for t in m.types})

    def ghost(self, ub):
        out = ub.copy()
        for tag in np.unique(self.m.bnd_tag):
            sel = self.m.bnd_tag == tag
            bc = self.bcs[int(tag)]
            if bc[0] == "state":
                out[sel] = self._ghost_state[int(tag)]
            elif bc[0] == "prescribed":
                x = self.m.flat(self.m.fpts_x)[self.m.bnd_g[sel]]
                w = np.asarray(bc[1](x), float)
                out[sel] = prim_to_cons(w[:, 0], w[:, 1:4], w[:, 4], self.gamma)
            elif bc[0] != "extrap":
                raise ValueError(f"unknown boundary condition {bc[0]}")
        return out

    def _split(self, arr, extra=()):
        """Global flux-point array -> per-type (n_e, n_f, ...) arrays."""
        m, out = self.m, {}
        for t in m.types:
            n = m.ne[t] * m.el[t].nfpts
            out[t] = arr[m.foff[t]:m.foff[t] + n].reshape(
                (m.ne[t], m.el[t].nfpts) + arr.shape[1:])
        return out

    # --- gradient path (NS) --------------------------------------------------
    def gradients(self, u, uf):
        m = self.m
        uc = np.empty_like(uf)
        l, r = m.pair_l, m.pair_r
        wl, wr = 0.5 - self.beta, 0.5 + self.beta
        uc[l] = uc[r] = wl * uf[l] + wr * uf[r]
        if len(m.bnd_g):
            ub = uf[m.bnd_g]
            uc[m.bnd_g] = wl * ub + wr * self.ghost(ub)
        du = self._split(uc - uf)
        grads = {}
        for t in m.types:
            el = m.el[t]
            gref = np.stack(
                [np.einsum("zv,evk->ezk", el.D[d], u[t])
                 + np.einsum("zf,efk->ezk", el.LIFT,
                             el.fpts_norm[None, :, d, None] * du[t])
                 for d in range(3)], axis=2)                 # (e, z, 3, 5)
            S, J = m.S_u[t], m.detJ[t]
            grads[t] = np.einsum("ezij,ezik->ezjk", S, gref) / J[..., None, None]
        return grads

    # --- the right-hand side ---------------------------------------------------
    def rhs(self, u):
        m, g = self.m, self.gamma
        ns = self.physics == "ns"
        uf = self.interp(u)
        grads = self.gradients(u, uf) if ns else None
        if ns:
            gf = m.flat({t: np.einsum("fz,ezjk->efjk", m.el[t].M0, grads[t])
                         for t in m.types})
        # Step 2: common normal flux at every flux point
        fc = np.zeros_like(uf)
        l, r = m.pair_l, m.pair_r
        n = m.fn_all[l]
        F = rusanov(uf[l], uf[r], n, g)
        vl, vr = 0.5 + self.beta, 0.5 - self.beta
        if ns:
            fv = (vl * viscous_flux(uf[l], gf[l], g, self.mu, self.pr)
                  + vr * viscous_flux(uf[r], gf[r], g, self.mu, self.pr))
            F = F - np.einsum("pj,pjk->pk", n, fv) + self.tau * (uf[l] - uf[r])
        fc[l] = m.fm_all[l][:, None] * F
        fc[r] = -m.fm_all[r][:, None] * F
        if len(m.bnd_g):
            b = m.bnd_g
            ub = uf[b]
            ug = self.ghost(ub)
            nb = m.fn_all[b]
            F = rusanov(ub, ug, nb, g)
            if ns:
                fv = (vl * viscous_flux(ub, gf[b], g, self.mu, self.pr)
                      + vr * viscous_flux(ug, gf[b], g, self.mu, self.pr))
                F = F - np.einsum("pj,pjk->pk", nb, fv) + self.tau * (ub - ug)
            fc[b] = m.fm_all[b][:, None] * F
        fc = self._split(fc)
        out = {}
        for t in m.types:
            el = m.el[t]
            if t in self.aa:                                 # Step 3, projected
                B, P, Sq = self.aa[t]
                uq = np.einsum("qz,ezk->eqk", B, u[t])
                f = euler_flux(uq, g)
                if ns:
                    gq = np.einsum("qz,ezjk->eqjk", B, grads[t])
                    f = f - viscous_flux(uq, gq, g, self.mu, self.pr)
                ftq = np.einsum("eqij,eqjk->eqik", Sq, f)
                ft = np.einsum("zq,eqik->ezik", P, ftq)
            else:
                f = euler_flux(u[t], g)                      # (e, z, 3, 5)
                if ns:
                    f = f - viscous_flux(u[t], grads[t], g, self.mu, self.pr)
                ft = np.einsum("ezij,ezjk->ezik", m.S_u[t], f)   # Step 3
            div = sum(np.einsum("zv,evk->ezk", el.D[d], ft[:, :, d])
                      for d in range(3))
            ff = np.einsum("fz,ezdk->efdk", el.M0, ft)
            fn = np.einsum("fd,efdk->efk", el.fpts_norm, ff)
            div = div + np.einsum("zf,efk->ezk", el.LIFT, fc[t] - fn)
            out[t] = -div / m.detJ[t][..., None]             # Step 5
        return out
