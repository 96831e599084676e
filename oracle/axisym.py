"""CPU oracle (test infrastructure) of the 3D-axisymmetric D2Q9 model of
Section 2.3.1 (Eq. Afi: BGK with forcing and the axisymmetric source H_i),
coupled to the same 0D boundaries as the 3D solver (Section 2.2).  Plain
numpy, FP64, one sub-step at a time in the order of Algorithm 1.

Only tests, the smoke check and the benchmark's CPU baseline use this module;
the product path is the CUDA library.

Coordinates: pseudo-Cartesian (x, r); node (x, j) sits at r = j + 1/2
(lattice units, dx = dt = 1); the symmetry axis r = 0 lies below row j = 0.
Node codes as in 3D: 0 fluid, 1 rigid wall, 2 + k node of 0D boundary k
(columns x = 0, sign +1, or x = nx - 1, sign -1; axis 0).

Readings (the printed h^(2) of Eq. AH1 is garbled, so the source is derived
from the axisymmetric incompressible Navier-Stokes equations that Eq. Afi
must recover, with rho0 = 1):

* mass source (the paper's h^(1)): m = -u_r / r, applied as
  S_i = (1 - 1/(2 tau)) w_i m with the pressure moment P = c_s^2 (sum f + m/2)
  (the half-step treatment of Guo's forcing applied to a mass source);
* momentum source (the role of h^(2)): the 2D lattice equations differ from
  the axisymmetric ones by
      g_x = nu (d_r u_x + d_x u_r) / r - u_x u_r / r
      g_r = 2 nu (d_r u_r - u_r / r) / r - u_r u_r / r,
  applied through the Guo forcing term (with any body force added); the
  strain rates are taken locally from the non-equilibrium stress,
  nu (d_a u_b + d_b u_a) = -(1 - 1/(2 tau)) Pi^neq_ab,
  Pi^neq = sum_i e_i e_i (f_i - f^eq_i(c_s^2 sum f, j)) (against the
  equilibrium of f's own moments: the Chapman-Enskog expansion of this
  scheme gives sum e e f^(1) = -tau c_s^2 (grad v + grad v^T)
  - (c_s^2 / 2) m I - (v g + g v) / 2, and the last two terms are exactly
  what f^eq(c_s^2 sum f, j) differs from f^eq(P, v) by, to first order),
  and u = j (unforced) inside the source;
* the axis is a mirror: a population that would come from below r = 0 is
  the mirrored population (e_r -> -e_r) of the node above it;
  flows with radial velocity (every source term active) are pinned by a
  manufactured steady solution in a periodic pipe (tests);
* rigid walls: halfway bounce-back; 0D boundaries: Eq. Non-equilibrium3 per
  link with the same source terms at x_f as the collision there; boundary
  flow Q = sum over the first fluid layer of 2 pi r n.j / sum f (area 2 pi r
  per node), Q_u = Q / A, mean pressure area-weighted.
"""
from __future__ import annotations

import numpy as np

from . import lv_step_ord, rcr_step_ord, smooth

CS2 = 1.0 / 3.0
PREF = CS2
# D2Q9 in (e_x, e_r)
EX = np.array([0, 1, -1, 0, 0, 1, -1, 1, -1])
ER = np.array([0, 0, 0, 1, -1, 1, -1, -1, 1])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
OPP = np.array([0, 2, 1, 4, 3, 6, 5, 8, 7])
MIR = np.array([0, 1, 2, 4, 3, 7, 8, 5, 6])      # e_r -> -e_r

BC_VELOCITY, BC_RCR, BC_LV, BC_PRESSURE = 0, 1, 2, 3


def feq(P, ux, ur):
    """He-Luo incompressible equilibrium (Eq. feq), arrays broadcast: (9, ...)."""
    eu = EX.reshape(-1, *([1] * np.ndim(P))) * ux + ER.reshape(-1, *([1] * np.ndim(P))) * ur
    usq = ux * ux + ur * ur
    w = W.reshape(-1, *([1] * np.ndim(P)))
    return w * (3.0 * P + 3.0 * eu + 4.5 * eu * eu - 1.5 * usq)


def guo(tau, ux, ur, gx, gr):
    """Guo forcing term (Eq. f) for force density (gx, gr) at velocity (ux, ur)."""
    sh = (-1,) + (1,) * np.ndim(ux)
    ex, er, w = EX.reshape(sh), ER.reshape(sh), W.reshape(sh)
    eu = ex * ux + er * ur
    eg = ex * gx + er * gr
    ug = ux * gx + ur * gr
    return (1.0 - 0.5 / tau) * w * (3.0 * (eg - ug) + 9.0 * eu * eg)


class AxiOracle:
    """One axisymmetric instance.  ``node``: (nr, nx) uint8 codes; ``bcs``:
    :class:`workloads.spec.Boundary` objects with axis 0; ``periodic_x`` and
    ``body_force`` are for the pins: a scalar is a uniform axial force per
    unit volume, a pair of (nr, nx) arrays a force field (g_x, g_r) given
    per node, added to the axisymmetric source like the scalar."""

    def __init__(self, node, tau, bcs=(), q_scale=1, periodic_x=False, body_force=0.0):
        self.node = np.asarray(node, dtype=np.uint8)
        self.nr, self.nx = self.node.shape
        self.tau = float(tau)
        self.nu = CS2 * (self.tau - 0.5)
        self.q_scale = int(q_scale)
        self.periodic_x = bool(periodic_x)
        if np.ndim(body_force) == 0:
            self.Gx, self.Gr = float(body_force), 0.0
        else:
            gx, gr = body_force
            self.Gx = np.array(gx, dtype=np.float64).reshape(self.nr, self.nx)
            self.Gr = np.array(gr, dtype=np.float64).reshape(self.nr, self.nx)
        self.r = (np.arange(self.nr) + 0.5)[:, None] * np.ones((1, self.nx))
        self.fluid = self.node == 0
        self.f = np.where(self.node != 1, 1.0, 0.0)[None] * W[:, None, None]
        self.step_n = 0
        self.bcs = []
        for k, b in enumerate(bcs):
            self.bcs.append(self._setup_bc(k, b))
        # pull table: population i of fluid node c comes from population
        # src_i of node src_c (bounce-back and mirror resolved; populations
        # from 0D boundary nodes are replaced by the link ghosts)
        di, dc, si, sc = [], [], [], []
        for j in range(self.nr):
            for x in range(self.nx):
                if not self.fluid[j, x]:
                    continue
                for i in range(9):
                    xs, js, ii, _ = self._src(x, j, i) if i else (x, j, 0, 0)
                    di.append(i)
                    dc.append(j * self.nx + x)
                    si.append(ii)
                    sc.append(js * self.nx + xs)
        self.pull = tuple(np.array(a, dtype=np.int64) for a in (di, dc, si, sc))
        self.wave = []
        self._macros()

    # -- set-up ---------------------------------------------------------
    def _src(self, x, j, i):
        """Pull source of direction i at node (x, j): (x', j', i', kind) with
        kind 0 node, 1 wall (bounce-back), 2 outside."""
        xs, js, ii = x - EX[i], j - ER[i], i
        if js < 0:                               # mirror at the axis
            js, ii = 0, MIR[i]
        if self.periodic_x:
            xs %= self.nx
        if xs < 0 or xs >= self.nx or js >= self.nr:
            return x, j, OPP[i], 1
        if self.node[js, xs] == 1:
            return x, j, OPP[i], 1
        return xs, js, ii, 0

    def _setup_bc(self, k, b):
        code = 2 + k
        nodes = [(x, j) for j in range(self.nr) for x in range(self.nx) if self.node[j, x] == code]
        node_index = {nd: a for a, nd in enumerate(nodes)}
        links = []   # (x_f, j_f, direction arriving at x_f, boundary node index)
        for j in range(self.nr):
            for x in range(self.nx):
                if not self.fluid[j, x]:
                    continue
                for i in range(1, 9):
                    xs, js, ii, kind = self._src(x, j, i)
                    if kind == 0 and self.node[js, xs] == code:
                        links.append((x, j, i, node_index[(xs, js)]))
        xf = sorted({(x, j) for x, j, _, _ in links}, key=lambda t: (t[1], t[0]))
        xfi = {c: a for a, c in enumerate(xf)}
        lk = np.array(links, dtype=np.int64).reshape(-1, 4)
        par = list(b.params) + [0.0] * (5 - len(b.params))
        if par[4] == 0.0:
            par[4] = 1.0
        st = dict(kind=int(b.kind), sign=int(b.sign), par=par, links=links,
                  lx=lk[:, 0], lj=lk[:, 1], li=lk[:, 2], lnode=lk[:, 3],
                  xf=xf, link_xfi=np.array([xfi[(x, j)] for x, j, _, _ in links], dtype=np.int64),
                  profile=None if b.profile is None else np.asarray(b.profile, dtype=np.float64),
                  etab=None if b.elastance is None else np.asarray(b.elastance, dtype=np.float64),
                  Pw=0.0, Pv=0.0, valve=0.0, Td=-1e300, Pstar=0.0, Q=0.0, Qu=0.0, Pbar=PREF,
                  v0=np.zeros((len(xf), 2)))
        if st["kind"] == BC_RCR:
            st["Pw"] = par[3]
        elif st["kind"] == BC_LV:
            st["Pv"] = par[3]
        return st

    # -- sub-steps --------------------------------------------------------
    def _macros(self):
        f = self.f
        sf = f.sum(axis=0)
        jx = np.tensordot(EX, f, axes=1)
        jr = np.tensordot(ER, f, axes=1)
        r = self.r
        m = -jr / r                                          # mass source (h^(1))
        P = CS2 * (sf + 0.5 * m)
        # the strain rates are read from f against the equilibrium of its own
        # moments (c_s^2 sum f, j): the first-order non-equilibrium stress
        # then equals -tau c_s^2 (grad v + grad v^T) alone, without the
        # isotropic -(c_s^2 / 2) m I of the mass source's half step (which a
        # comparison with f^eq(P, j) would leave on the diagonal)
        fe = feq(CS2 * sf, jx, jr)
        dn = f - fe
        pxr = np.tensordot(EX * ER, dn, axes=1)
        prr = np.tensordot(ER * ER, dn, axes=1)
        k = 1.0 - 0.5 / self.tau
        gx = -k * pxr / r - jx * jr / r + self.Gx
        gr = -k * prr / r - 2.0 * self.nu * jr / (r * r) - jr * jr / r + self.Gr
        z = ~self.fluid
        for a in (sf, jx, jr, m, P, gx, gr):
            a[z] = 0.0
        self.sf, self.jx, self.jr, self.m, self.P, self.gx, self.gr = sf, jx, jr, m, P, gx, gr
        self.vx = jx + 0.5 * gx
        self.vr = jr + 0.5 * gr

    def _fluxes(self):
        for b in self.bcs:
            Q = A = Ps = 0.0
            for (x, j) in b["xf"]:
                a = 2.0 * np.pi * (j + 0.5)
                Q += a * b["sign"] * self.jx[j, x] / self.sf[j, x]
                Ps += a * self.P[j, x]
                A += a
            b["Q"] = Q
            b["Qu"] = Q / A if self.q_scale else Q
            b["Pbar"] = Ps / A

    def _evolve_0d(self):
        n = self.step_n
        for b in self.bcs:
            par = b["par"]
            if b["kind"] == BC_RCR:
                b["Pw"], b["Pstar"] = rcr_step_ord(b["Pw"], -b["Qu"], par[0], par[1], par[2], int(par[4]))
            elif b["kind"] == BC_PRESSURE:
                b["Pstar"] = par[0]
            elif b["kind"] == BC_LV:
                T = b["etab"].shape[0]
                E, Ed = b["etab"][n % T]
                E1, Ed1 = b["etab"][(n + 1) % T]
                b["Pv"], b["valve"], b["Td"], closed = lv_step_ord(
                    b["Pv"], b["valve"], b["Td"], n, E, Ed, E1, Ed1, int(par[4]), b["Qu"],
                    b["Pbar"] - PREF, par[1])
                if closed:
                    for a, (x, j) in enumerate(b["xf"]):
                        b["v0"][a] = (self.vx[j, x], self.vr[j, x])
                b["Pstar"] = b["Pv"]

    def _ghosts(self):
        """Eq. Non-equilibrium3 for every link: the population arriving at x_f."""
        tn1 = float(self.step_n + 1)
        out = []
        for b in self.bcs:
            ptype = b["kind"] in (BC_RCR, BC_PRESSURE) or (b["kind"] == BC_LV and b["valve"] != 0.0)
            x, j, i = b["lx"], b["lj"], b["li"]
            Pf, vx, vr = self.P[j, x], self.vx[j, x], self.vr[j, x]
            if ptype:
                Ps, sx, sr = PREF + b["Pstar"] + 0 * Pf, vx, vr
            elif b["kind"] == BC_VELOCITY:
                pr = b["profile"][b["lnode"]]
                w = b["par"][0]
                Ps = Pf
                sx = b["sign"] * (pr[:, 0] + pr[:, 1] * np.cos(w * tn1) - pr[:, 2] * np.sin(w * tn1))
                sr = 0 * Pf
            else:
                S = smooth(tn1, b["Td"], b["par"][2])
                v0 = b["v0"][b["link_xfi"]]
                Ps, sx, sr = Pf, v0[:, 0] * S, v0[:, 1] * S
            n = np.arange(x.size)
            F = guo(self.tau, vx, vr, self.gx[j, x], self.gr[j, x]) + \
                (1.0 - 0.5 / self.tau) * W[:, None] * self.m[j, x]
            g = (feq(Ps, sx, sr)[i, n] + (1.0 - 1.0 / self.tau) * (self.f[i, j, x] - feq(Pf, vx, vr)[i, n])
                 + F[i, n])
            out.append((i, j, x, g))
        return out

    def _collide(self):
        fe = feq(self.P, self.vx, self.vr)
        F = guo(self.tau, self.vx, self.vr, self.gx, self.gr) + (1.0 - 0.5 / self.tau) * W[:, None, None] * self.m
        post = self.f - (self.f - fe) / self.tau + F
        return np.where(self.fluid[None], post, self.f)

    def _stream(self, post, ghosts):
        di, dc, si, sc = self.pull
        new = self.f.reshape(9, -1).copy()
        new[di, dc] = post.reshape(9, -1)[si, sc]
        new = new.reshape(9, self.nr, self.nx)
        for i, j, x, g in ghosts:
            new[i, j, x] = g
        self.f = new

    def _log(self):
        row = [float(self.step_n)]
        for b in self.bcs:
            state = b["Pw"] if b["kind"] == BC_RCR else (b["Pv"] if b["kind"] == BC_LV else b["Pstar"])
            row += [b["Qu"], b["Pbar"] - PREF, state, b["valve"]]
        self.wave.append(row)

    def step(self, n: int = 1):
        for _ in range(n):
            self._macros()
            self._fluxes()
            self._evolve_0d()
            ghosts = self._ghosts()
            post = self._collide()
            self._stream(post, ghosts)
            self._log()
            self.step_n += 1
        self._macros()

    # -- read-out -----------------------------------------------------------
    def fields(self):
        """P, u_x, u_r (fluid velocity j + g/2) of f(t_n); zero off the fluid."""
        self._macros()
        return self.P.copy(), self.vx.copy(), self.vr.copy()

    def populations(self):
        return self.f.copy()

    def set_populations(self, f):
        self.f = np.array(f, dtype=np.float64).reshape(9, self.nr, self.nx)
        self._macros()

    def waves(self):
        return np.array(self.wave)

    def state_0d(self, k):
        b = self.bcs[k]
        return dict(Pw=b["Pw"], Pv=b["Pv"], valve=b["valve"], Td=b["Td"], Qu=b["Qu"], Pbar=b["Pbar"])
