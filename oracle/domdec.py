"""Unbalanced domain decomposition (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

What is computed, in the paper's order:
  * Grids, basic cells and the composite partitions A (aligned) and B
    (shifted by one basic cell, boundary cells clipped to the image), and the
    2^d staggered sub-batches of each partition (Definition 2.4; Section 5.3,
    'Basic and composite partitions' and 'staggered strategy and batching').
  * The plan is stored through its basic-cell Y-marginals nu_i on bounding
    boxes, truncated below ``thr`` (Section 2.3 end; Section 5.1 'Computing
    and handling nu_{-J}'; Section 5.3 'Stopping criterion and measure
    truncation').
  * One parallel DomDec iteration (Algorithm 4) per sub-batch: every cell J
    solves its subproblem from the same state with nu_{-J} = P_Y pi - nu_J
    restricted to the box B_J, then GetWeights (greedy / safe / swift,
    Eq. GWFast and Proposition 4.3) picks theta and the cell plans are mixed.
    ``staggered`` = swift on each sub-batch (Section 4.4).
  * Sequential DomDec (Algorithm 3): cells one at a time, theta = 1.

Readings where the paper leaves a choice (each listed in the design notes):
  R1  nu_{-J}/nu is clamped at 0 (round-off can make P_Y pi - nu_J negative).
  R2  The cell problem's Y is the bounding box B_J of the member boxes; the
      new cell plan is zero outside it.
  R3  The score of a mixed plan is tracked, not re-instantiated: per basic
      cell the transport cost C_i = <c, pi_i> and the entropy
      H_i = KL(pi_i | mu_i x nu) are mixed linearly (exact for C_i, an upper
      bound for H_i by convexity); the marginal terms are evaluated exactly
      from P_X pi and P_Y pi, which mix linearly.  Tracked score
      E_hat = sum_i (C_i + eps H_i) + lam KL(P_X pi|mu) + lam KL(P_Y pi|nu).
  R4  swift: theta = 1 if E(1) <= E(1/|b|) (+ 1e-12 |E_hat| tie slack) or, with
      leniency tau > 0, if E(1) <= (1 + tau) E_hat; else theta = 1/|b|.
  R5  Sub-batches run in the order (0,0), (0,1), (1,0), (1,1) of the
      composite index parities; sweep k = 0, 2, 4, ... uses A, odd k uses B.
  R6  After mixing, nu_i(y) < thr is set to 0 and the box shrinks to the
      remaining support; C_i, H_i and P_X pi are not corrected for the
      truncated mass (at most thr per truncated entry).
  R7  The cell Sinkhorn warm-starts from the stored alpha on X_J and the
      stored alpha is replaced by the cell's final alpha whatever theta is.
"""
from __future__ import annotations

import numpy as np

from . import uot
from .cell import cell_sinkhorn

INF = float("inf")


# =================================================================== geometry
class Geometry:
    """X = Y = {0..N-1}^d pixels with spacing h = 1/N; basic cells are s^d
    blocks; composite cells group 2^d basic cells."""

    def __init__(self, N, s, d=2):
        if N % (2 * s):
            raise ValueError("N must be divisible by 2s")
        self.N, self.s, self.d = int(N), int(s), int(d)
        self.h = 1.0 / N
        self.n = N ** d
        self.nb = N // s
        self.nbasic = self.nb ** d
        self.pix = uot.grid_index(N, d)
        bidx = self.pix // s
        self.basic_of_pixel = np.ravel_multi_index(tuple(bidx.T), (self.nb,) * d)
        order = np.argsort(self.basic_of_pixel, kind="stable")
        cuts = np.searchsorted(self.basic_of_pixel[order], np.arange(self.nbasic + 1))
        self.basic_pixels = [order[cuts[i]:cuts[i + 1]] for i in range(self.nbasic)]
        self.parts = {"A": self._partition(0), "B": self._partition(1)}

    def box_flat(self, lo, hi):
        """Flat (row-major) pixel indices of the box [lo, hi)."""
        rng = [np.arange(a, b) for a, b in zip(lo, hi)]
        if any(len(r) == 0 for r in rng):
            return np.zeros(0, np.int64)
        mesh = np.meshgrid(*rng, indexing="ij")
        return np.ravel_multi_index(tuple(m.ravel() for m in mesh), (self.N,) * self.d)

    def _partition(self, off):
        d, s, nb, N = self.d, self.s, self.nb, self.N
        nc = nb // 2 + off
        cells = []
        for P in np.ndindex(*((nc,) * d)):
            P = np.array(P)
            lo_b = 2 * P - off
            members = []
            for a in np.ndindex(*((2,) * d)):
                I = lo_b + np.array(a)
                if np.all(I >= 0) and np.all(I < nb):
                    members.append(int(np.ravel_multi_index(tuple(I), (nb,) * d)))
            xlo = np.maximum(0, s * lo_b)
            xhi = np.minimum(N, s * (lo_b + 2))
            sub = 0
            for k in range(d):
                sub = 2 * sub + int(P[k] % 2)
            cells.append(dict(P=tuple(int(p) for p in P), members=members,
                              xlo=xlo, xhi=xhi, X=self.box_flat(xlo, xhi), sub=sub))
        return cells


# ====================================================================== state
class State:
    """DomDec state: alpha (stitched X-potential, the warm start), P_X pi,
    P_Y pi, and per basic cell a Y-box [lo, hi) with the values of nu_i there,
    C_i and H_i.  ``pi`` optionally keeps the dense plan (small N only) so that
    the tracked score can be compared with the exact one."""

    def __init__(self, geo, mu, nu, eps, lam, thr):
        self.geo = geo
        self.mu = np.asarray(mu, np.float64).ravel()
        self.nu = np.asarray(nu, np.float64).ravel()
        self.eps, self.lam, self.thr = float(eps), float(lam), float(thr)
        n, nbasic, d = geo.n, geo.nbasic, geo.d
        self.alpha = np.zeros(n)
        self.PX = np.zeros(n)
        self.PY = np.zeros(n)
        self.lo = np.zeros((nbasic, d), np.int64)
        self.hi = np.zeros((nbasic, d), np.int64)
        self.vals = [np.zeros((0,) * d) for _ in range(nbasic)]
        self.Cc = np.zeros(nbasic)
        self.Hh = np.zeros(nbasic)
        self.pi = None

    # ---- helpers
    def embed(self, i, lo, hi):
        """nu_i as a dense array over the box [lo, hi) (which must contain
        the box of nu_i)."""
        out = np.zeros(tuple(hi - lo))
        if self.vals[i].size:
            sl = tuple(slice(a - b, c - b) for a, b, c in zip(self.lo[i], lo, self.hi[i]))
            out[sl] = self.vals[i]
        return out

    def set_basic(self, i, vals, lo):
        """Truncate values below thr to 0 and store the tight box (R6)."""
        v = np.where(vals < self.thr, 0.0, vals)
        nz = np.nonzero(v)
        if len(nz[0]) == 0:
            self.lo[i] = lo
            self.hi[i] = lo
            self.vals[i] = np.zeros((0,) * self.geo.d)
            return
        a = np.array([x.min() for x in nz])
        b = np.array([x.max() + 1 for x in nz])
        self.lo[i] = lo + a
        self.hi[i] = lo + b
        self.vals[i] = v[tuple(slice(p, q) for p, q in zip(a, b))].copy()

    def recompute_PY(self):
        """P_Y pi = sum_i nu_i (Section 5.1, 'Computing and handling nu_{-J}')."""
        g = self.geo
        PY = np.zeros(g.n)
        for i in range(g.nbasic):
            if self.vals[i].size:
                PY[g.box_flat(self.lo[i], self.hi[i])] += self.vals[i].ravel()
        self.PY = PY

    def zero_truncated_plan_entries(self, i):
        """Keep the dense plan consistent with a truncated nu_i."""
        if self.pi is None:
            return
        g = self.geo
        full = np.zeros(g.n)
        if self.vals[i].size:
            full[g.box_flat(self.lo[i], self.hi[i])] = self.vals[i].ravel()
        rows = g.basic_pixels[i]
        self.pi[np.ix_(rows, np.flatnonzero(full == 0))] = 0.0

    def box_entries(self):
        return int(sum(v.size for v in self.vals))


def full_cost(geo):
    return uot.sq_cost(geo.pix, geo.pix, geo.h)


def init_product(geo, mu, nu, eps, lam, thr=1e-15, track_plan=False):
    """Initial plan pi0 = mu x nu (Section 4.1, toy problem): nu_i = |mu_i| nu
    on the full grid, P_X = |nu| mu, alpha = 0, H_i = 0 and
    C_i = sum_{x in X_i, y} c(x,y) mu(x) nu(y)."""
    st = State(geo, mu, nu, eps, lam, thr)
    N, d = geo.N, geo.d
    full_lo = np.zeros(d, np.int64)
    nu_img = st.nu.reshape((N,) * d)
    for i in range(geo.nbasic):
        rows = geo.basic_pixels[i]
        mi = st.mu[rows].sum()
        st.set_basic(i, mi * nu_img, full_lo)
        C = uot.sq_cost(geo.pix[rows], geo.pix, geo.h)
        st.Cc[i] = float(np.sum(C * st.mu[rows, None] * st.nu[None, :]))
        st.Hh[i] = 0.0
    st.PX = st.mu * st.nu.sum()
    st.recompute_PY()
    if track_plan:
        st.pi = st.mu[:, None] * st.nu[None, :]
        for i in range(geo.nbasic):
            st.zero_truncated_plan_entries(i)
    return st


def init_from_duals(geo, mu, nu, alpha, beta, eps0, eps, lam, thr=1e-15,
                    track_plan=False):
    """Initial plan pi = exp((alpha (+) beta - c)/eps0) mu x nu, e.g. from a
    global Sinkhorn warm start (Section 5.3, 'Sinkhorn warm start'):
    nu_i = sum_{x in X_i} pi(x, .) truncated; C_i, H_i from the full plan."""
    st = State(geo, mu, nu, eps, lam, thr)
    C = full_cost(geo)
    pi = uot.plan(np.asarray(alpha, np.float64), np.asarray(beta, np.float64),
                  C, st.mu, st.nu, eps0)
    N, d = geo.N, geo.d
    full_lo = np.zeros(d, np.int64)
    logratio = (alpha[:, None] + beta[None, :] - C) / eps0
    for i in range(geo.nbasic):
        rows = geo.basic_pixels[i]
        st.set_basic(i, pi[rows].sum(0).reshape((N,) * d), full_lo)
        st.Cc[i] = float(np.sum(C[rows] * pi[rows]))
        st.Hh[i] = float(np.sum(pi[rows] * logratio[rows] - pi[rows])
                         + st.mu[rows].sum() * st.nu.sum())
    st.PX = pi.sum(1)
    st.alpha = np.array(alpha, np.float64)
    st.recompute_PY()
    if track_plan:
        st.pi = pi.copy()
        for i in range(geo.nbasic):
            st.zero_truncated_plan_entries(i)
    return st


# ====================================================================== score
def tracked_score(st, Cc=None, Hh=None, PX=None, PY=None):
    """E_hat = sum_i (C_i + eps H_i) + lam KL(P_X|mu) + lam KL(P_Y|nu)  (R3;
    the split of the score over cells is Eq. domdec-score-decomp-unbalanced)."""
    Cc = st.Cc if Cc is None else Cc
    Hh = st.Hh if Hh is None else Hh
    PX = st.PX if PX is None else PX
    PY = st.PY if PY is None else PY
    return float(np.sum(Cc) + st.eps * np.sum(Hh)
                 + st.lam * uot.kl(PX, st.mu) + st.lam * uot.kl(np.maximum(PY, 0.0), st.nu))


def exact_score(st):
    """E(pi) of the dense plan (Eq. unbalanced-problem); needs track_plan."""
    return uot.primal_score(st.pi, full_cost(st.geo), st.mu, st.nu, st.eps, st.lam)


def score_terms(st):
    """(E_hat, sum_i(C_i + eps H_i), lam KL(P_X|mu), lam KL(P_Y|nu), |P_Y|)."""
    loc = float(np.sum(st.Cc) + st.eps * np.sum(st.Hh))
    kx = st.lam * uot.kl(st.PX, st.mu)
    ky = st.lam * uot.kl(np.maximum(st.PY, 0.0), st.nu)
    return loc + kx + ky, loc, kx, ky, float(st.PY.sum())


# ================================================================ cell solves
def cell_problem(st, cell, margin=0):
    """B_J = bounding box of the member boxes (widened by margin, clipped);
    nu_J on B_J; rho = max(0, P_Y - nu_J)/nu on B_J (R1, R2)."""
    g = st.geo
    mem = [i for i in cell["members"] if st.vals[i].size]
    if not mem:
        return None
    lo = np.min([st.lo[i] for i in mem], axis=0) - margin
    hi = np.max([st.hi[i] for i in mem], axis=0) + margin
    lo = np.maximum(lo, 0)
    hi = np.minimum(hi, g.N)
    Y = g.box_flat(lo, hi)
    nuJ = np.zeros(tuple(hi - lo))
    for i in cell["members"]:
        if st.vals[i].size:
            nuJ += st.embed(i, lo, hi)
    rho = np.maximum(0.0, st.PY[Y] - nuJ.ravel()) / st.nu[Y]
    return dict(lo=lo, hi=hi, Y=Y, rho=rho)


def balance_factors(st, X, Y, C, beta, pi, rows):
    """Balancing step (Section 5.3, 'Balancing', Eq. balancing) for one cell.

    One more X-half from the final beta gives alpha' and the X-marginal of
    the next plan, mu_bar = e^{-alpha'/lam} mu_J (mu_J itself for lam = inf);
    the targets are m_i = mu_bar(X_i) |nu_J| / mu_bar(X_J) with |nu_J| the
    mass of the new cell plan.  The paper asks for a horizontal shift of mass
    between the basic cells (y fixed) with |nu_i| = m_i and nu_J preserved,
    without fixing the rule.  Reading: donors (|nu_i| > m_i) give the same
    fraction of their marginal at every y; the donated field
    D(y) = sum_d (|nu_d| - m_d) nu_d(y) / |nu_d| is shared at every y among the
    receivers in proportion to their deficits, and a receiver's new mass at y
    follows its own plan row (the new cell plan is positive on X_J x B_J).
    So the balanced plan is pi_i(x, y) rho_i(y) with
      rho_d = m_d / |nu_d|,   rho_r(y) = 1 + D(y) (m_r - |nu_r|) / (E nu_r(y)),
    E = sum_d (|nu_d| - m_d); nu_J is preserved at every y and |nu_i| = m_i.
    Returns {i: rho_i (n_y,)}; all ones when nothing is to move."""
    eps, lam = st.eps, st.lam
    logmu = np.log(st.mu[X])
    if np.isinf(lam):
        mubar = st.mu[X]
    else:
        a2 = uot.x_half(beta, C, st.nu[Y], eps, lam)
        mubar = np.exp(logmu - a2 / lam)
    nut = {i: pi[r].sum(0) for i, r in rows.items()}
    mass = {i: float(v.sum()) for i, v in nut.items()}
    mJ = sum(mass.values())
    m = {i: float(mubar[r].sum()) * mJ / float(mubar.sum()) for i, r in rows.items()}
    exc = {i: mass[i] - m[i] for i in rows}
    E = sum(e for e in exc.values() if e > 0)
    rho = {i: np.ones(len(Y)) for i in rows}
    if not E > 0:
        return rho
    D = np.zeros(len(Y))
    for i, e in exc.items():
        if e > 0:
            D += (e / mass[i]) * nut[i]
            rho[i] = np.full(len(Y), m[i] / mass[i])
    for i, e in exc.items():
        if e < 0:
            with np.errstate(divide="ignore", invalid="ignore"):
                add = np.where(nut[i] > 0, D * (-e / E) / nut[i], 0.0)
            rho[i] = 1.0 + add
    return rho


def solve_cell(st, cell, prob, err=2e-5, maxit=2000, ti=False, balance=False):
    """Solve the cell subproblem and return the new cell plan's data: final
    duals, P_X of the new plan on X_J, and per member basic cell its new
    Y-marginal on B_J, C_i and H_i (H_i via log(pi/(mu nu)) =
    (alpha+beta-c)/eps for the diagonal scaling, Eq. diagonal-scaling).
    With ``balance`` the plan is first balanced (balance_factors)."""
    g = st.geo
    X, Y = cell["X"], prob["Y"]
    C = uot.sq_cost(g.pix[X], g.pix[Y], g.h)
    res = cell_sinkhorn(st.mu[X], st.nu[Y], prob["rho"], C, st.eps, st.lam,
                        st.alpha[X], err, maxit, ti)
    pi = uot.plan(res.alpha, res.beta, C, st.mu[X], st.nu[Y], st.eps)
    logratio = (res.alpha[:, None] + res.beta[None, :] - C) / st.eps
    shape = tuple(prob["hi"] - prob["lo"])
    bop = g.basic_of_pixel[X]
    rows = {i: bop == i for i in cell["members"]}
    px = res.px
    if balance:
        rho = balance_factors(st, X, Y, C, res.beta, pi, rows)
        for i, r in rows.items():
            pi[r] = pi[r] * rho[i][None, :]
            with np.errstate(divide="ignore"):
                logratio[r] = logratio[r] + np.log(rho[i])[None, :]
        px = pi.sum(1)
    nut, Ct, Ht = {}, {}, {}
    nu_tot = st.nu.sum()
    for i, r in rows.items():
        nut[i] = pi[r].sum(0).reshape(shape)
        Ct[i] = float(np.sum(C[r] * pi[r]))
        pr = pi[r]
        Ht[i] = float(np.sum(np.where(pr > 0, pr * logratio[r], 0.0) - pr) + st.mu[X][r].sum() * nu_tot)
    return dict(alpha=res.alpha, beta=res.beta, px=px, nut=nut, Ct=Ct, Ht=Ht,
                iters=res.iters, converged=res.converged, gap=res.gap, pi=pi)


# ============================================================ GetWeights, mix
def mixed_quantities(st, batch, probs, sols, theta):
    """Bookkeeping quantities of sum_J (1-theta) pi_J + theta pi~_J before
    truncation: (C, H, P_X, P_Y)."""
    Cc, Hh, PX, PY = st.Cc.copy(), st.Hh.copy(), st.PX.copy(), st.PY.copy()
    for cell, prob, sol in zip(batch, probs, sols):
        if prob is None:
            continue
        X = cell["X"]
        PX[X] = (1 - theta) * st.PX[X] + theta * sol["px"]
        for i in cell["members"]:
            Cc[i] = (1 - theta) * st.Cc[i] + theta * sol["Ct"][i]
            Hh[i] = (1 - theta) * st.Hh[i] + theta * sol["Ht"][i]
            old = st.embed(i, prob["lo"], prob["hi"])
            PY[prob["Y"]] += theta * (sol["nut"][i] - old).ravel()
    return Cc, Hh, PX, PY


LINE_ITERS = 48      # cap on steps of the GetWeights_line root search
LINE_GTOL = 1e-12    # stop when |E'| <= LINE_GTOL * (sum of the magnitudes of its terms)
LINE_XTOL = 1e-12    # ... or when the bracket is this narrow
LINE_PFLOOR = 1e-300  # floor of a mixed marginal inside the logarithm


def line_search(st, batch, probs, sols, lo):
    """GetWeights_line (Proposition 4.3, item 4): the zeta in [lo, 1] with the
    largest decrement of the score of sum_J (1-zeta) pi_J + zeta pi~_J.

    Reading (the paper does not say how the search is done): the score is the
    tracked E_hat (R3).  Along zeta, C and H mix linearly and so do the
    marginals, hence
      E'(zeta)  = L + lam <dX, log(P_X(zeta)/mu)> + lam <dY, log(P_Y(zeta)/nu)>,
      E''(zeta) = lam <dX^2, 1/P_X(zeta)> + lam <dY^2, 1/P_Y(zeta)> >= 0,
    with L = sum_i (C~_i - C_i) + eps (H~_i - H_i) and dX, dY the marginal
    changes at zeta = 1.  E_hat is convex in zeta, so the minimiser on [lo, 1]
    is 1 if E'(1) <= 0, lo if E'(lo) >= 0, and otherwise the root of E' in the
    bracket [lo, 1]: Newton steps from zeta = 1, replaced by the bracket's
    midpoint when a step leaves the bracket or when the bracket has not halved
    over the last two steps (a Newton step can be tiny far from the root where
    a mixed marginal nearly vanishes); stop when |E'| <= LINE_GTOL times the sum
    of the magnitudes of its terms, when the bracket is narrower than
    LINE_XTOL, or after LINE_ITERS steps.  Returns the last point evaluated."""
    Cg, Hg, PXg, PYg = mixed_quantities(st, batch, probs, sols, 1.0)
    L = float(np.sum(Cg - st.Cc) + st.eps * np.sum(Hg - st.Hh))
    dX = PXg - st.PX
    dY = PYg - st.PY
    mx, my = dX != 0.0, dY != 0.0
    p0x, dx, mux = st.PX[mx], dX[mx], st.mu[mx]
    p0y, dy, nuy = st.PY[my], dY[my], st.nu[my]

    def derivs(z):
        px = np.maximum(p0x + z * dx, LINE_PFLOOR)
        py = np.maximum(p0y + z * dy, LINE_PFLOOR)
        tx = dx * np.log(px / mux)
        ty = dy * np.log(py / nuy)
        g = L + st.lam * float(np.sum(tx)) + st.lam * float(np.sum(ty))
        h = st.lam * float(np.sum(dx * dx / px)) + st.lam * float(np.sum(dy * dy / py))
        scale = abs(L) + st.lam * float(np.sum(np.abs(tx))) + st.lam * float(np.sum(np.abs(ty)))
        return g, h, scale

    g, h, _ = derivs(1.0)
    if g <= 0.0:
        return 1.0
    if derivs(lo)[0] >= 0.0:
        return lo
    a, b, z = lo, 1.0, 1.0
    widths = [np.inf, np.inf]
    for _ in range(LINE_ITERS):
        zn = z - g / h if h > 0.0 else a
        if not (a < zn < b) or (b - a) > 0.5 * widths[-2]:
            zn = 0.5 * (a + b)
        z = zn
        g, h, scale = derivs(z)
        if g > 0.0:
            b = z
        else:
            a = z
        widths.append(b - a)
        if abs(g) <= LINE_GTOL * scale or b - a <= LINE_XTOL:
            break
    return z


def get_weights(st, batch, probs, sols, strategy, tau):
    """GetWeights for a batch (Eq. GWFast, Proposition 4.3; swift per
    sub-batch for ``staggered``; ``line`` = GetWeights_line).  Returns
    (theta, E_hat, E(1), E(safe))."""
    nb = sum(p is not None for p in probs)
    th_safe = 1.0 / max(nb, 1)
    E0 = tracked_score(st)
    if strategy == "greedy":
        return 1.0, E0, None, None
    if strategy == "safe":
        return th_safe, E0, None, None
    Eg = tracked_score(st, *mixed_quantities(st, batch, probs, sols, 1.0))
    Es = tracked_score(st, *mixed_quantities(st, batch, probs, sols, th_safe))
    if strategy in ("line", "staggered_line"):
        return line_search(st, batch, probs, sols, th_safe), E0, Eg, Es
    if Eg <= Es + 1e-12 * abs(E0) or (tau > 0 and Eg <= (1 + tau) * E0):
        return 1.0, E0, Eg, Es
    return th_safe, E0, Eg, Es


def apply_step(st, batch, probs, sols, theta):
    """pi' = sum_J (1-theta) pi_J + theta pi~_J (Algorithm 4, last line), then
    truncation and box refresh (R6, R7), then P_Y pi = sum_i nu_i."""
    g = st.geo
    for cell, prob, sol in zip(batch, probs, sols):
        if prob is None:
            continue
        X = cell["X"]
        st.PX[X] = (1 - theta) * st.PX[X] + theta * sol["px"]
        st.alpha[X] = sol["alpha"]
        if st.pi is not None:
            new = np.zeros((len(X), g.n))
            new[:, prob["Y"]] = sol["pi"]
            st.pi[X] = (1 - theta) * st.pi[X] + theta * new
        for i in cell["members"]:
            old = st.embed(i, prob["lo"], prob["hi"])
            st.set_basic(i, (1 - theta) * old + theta * sol["nut"][i], prob["lo"])
            st.Cc[i] = (1 - theta) * st.Cc[i] + theta * sol["Ct"][i]
            st.Hh[i] = (1 - theta) * st.Hh[i] + theta * sol["Ht"][i]
            st.zero_truncated_plan_entries(i)
    st.recompute_PY()


# ===================================================================== sweeps
def batches_of(st, which, strategy):
    cells = st.geo.parts[which]
    if strategy in ("staggered", "staggered_line"):
        nsub = 2 ** st.geo.d
        out = [[c for c in cells if c["sub"] == b] for b in range(nsub)]
        return [b for b in out if b]
    return [cells]


def sweep(st, which, strategy="staggered", tau=0.0, err=2e-5, maxit=2000, margin=0, ti=False,
          balance=False):
    """One parallel DomDec iteration over partition ``which`` (Algorithm 4;
    for ``staggered`` once per sub-batch, in sub-batch order).  Returns one
    log record per batch."""
    log = []
    for batch in batches_of(st, which, strategy):
        probs = [cell_problem(st, c, margin) for c in batch]
        sols = [None if p is None else solve_cell(st, c, p, err, maxit, ti, balance)
                for c, p in zip(batch, probs)]
        theta, E0, Eg, Es = get_weights(st, batch, probs, sols, strategy, tau)
        apply_step(st, batch, probs, sols, theta)
        log.append(dict(theta=theta, E0=E0, Eg=Eg, Es=Es, ncell=len(batch),
                        iters=[s["iters"] for s in sols if s is not None],
                        converged=[s["converged"] for s in sols if s is not None]))
    return log


def sequential_sweep(st, which, err=2e-5, maxit=2000, margin=0, ti=False, balance=False):
    """Sequential DomDec iteration (Algorithm 3): cells in partition order,
    each solved from the current state and accepted with theta = 1."""
    iters = []
    for cell in st.geo.parts[which]:
        prob = cell_problem(st, cell, margin)
        if prob is None:
            continue
        sol = solve_cell(st, cell, prob, err, maxit, ti, balance)
        apply_step(st, [cell], [prob], [sol], 1.0)
        iters.append(sol["iters"])
    return iters


def run(st, n_sweeps, strategy="staggered", tau=0.0, err=2e-5, maxit=2000,
        margin=0, first=0, record=None, ti=False, balance=False):
    """Alternate A and B sweeps (Algorithm 2): sweep k uses A for even
    first+k, B otherwise.  ``record(k, st, log)`` is called after each sweep."""
    logs = []
    for k in range(n_sweeps):
        which = "A" if (first + k) % 2 == 0 else "B"
        if strategy == "sequential":
            lg = sequential_sweep(st, which, err, maxit, margin, ti, balance)
        else:
            lg = sweep(st, which, strategy, tau, err, maxit, margin, ti, balance)
        logs.append(lg)
        if record is not None:
            record(k, st, lg)
    return logs


# ============================================================== certificates
def y_half_global(st, alpha, chunk=4096):
    """beta* = -kappa log int exp((alpha - c)/eps) dmu over the whole grid
    (global Y-half with nu_- = 0, Eq. sinkhorn-iters-ot), chunked over y."""
    g = st.geo
    out = np.empty(g.n)
    logmu = np.log(st.mu)
    for a in range(0, g.n, chunk):
        ys = np.arange(a, min(g.n, a + chunk))
        C = uot.sq_cost(g.pix, g.pix[ys], g.h)
        out[ys] = -uot.kappa(st.eps, st.lam) * uot.lse((alpha[:, None] - C) / st.eps
                                                       + logmu[:, None], 0)
    return out


def dual_value(st, alpha, beta, chunk=4096):
    """D(alpha, beta | 0) (Eq. dual-problem, D_i = lam KL), chunked over y."""
    g = st.geo
    ent = 0.0
    for a in range(0, g.n, chunk):
        ys = np.arange(a, min(g.n, a + chunk))
        C = uot.sq_cost(g.pix, g.pix[ys], g.h)
        e = np.exp((alpha[:, None] + beta[None, ys] - C) / st.eps)
        ent += float(np.sum((1.0 - e) * st.mu[:, None] * st.nu[None, ys]))
    return (st.eps * ent - uot.conj_term(alpha, st.mu, st.lam)
            - uot.conj_term(beta, st.nu, st.lam))


def pd_certificate(st):
    """Primal E_hat (an upper bound of the score of the stored plan), dual
    D(alpha, beta*) with the stitched alpha and beta* from one global Y-half,
    and the relative gap (E_hat - D)/|D| (Section 5.3, 'Solution quality')."""
    beta = y_half_global(st, st.alpha)
    D = dual_value(st, st.alpha, beta)
    P = tracked_score(st)
    return P, D, (P - D) / abs(D), beta


def marginal_errors(st, beta):
    """L1 X- and Y-marginal errors |P_X - e^{-alpha/lam} mu|_1 and
    |P_Y - e^{-beta/lam} nu|_1 (Section 5.3, 'Solution quality')."""
    ex = float(np.sum(np.abs(st.PX - np.exp(-st.alpha / st.lam) * st.mu)))
    ey = float(np.sum(np.abs(st.PY - np.exp(-beta / st.lam) * st.nu)))
    return ex, ey
