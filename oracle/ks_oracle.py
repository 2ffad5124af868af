"""Plain, slow FP64 CPU oracle for the adjoint-based variational tau-descent of KS loops.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this module.  The
product path never calls it and shares no code with it: every transform here is a naive
dense DFT (matrix products over the paper's signed mode ranges), with no FFT library, no
half-spectrum tricks and no blocking or fusion.

Paper: Azimi, Ashtari & Schneider, "Adjoint-based variational method for constructing
periodic orbits of high-dimensional chaotic systems" (arXiv:2007.06427).

What is computed, in the paper's order and notation (KS with nu = 1):

* a loop is l = [u(x, s); T] on [0, L) x [0, 1), both directions periodic (Sec. 2,
  Eq. loop_def);
* residual r = -(1/T) u_s - u u_x - u_xx - u_xxxx (Sec. 4.1, Eq. KS_R);
* cost J = int_0^1 int_0^L r^2 dx ds (Sec. 2, Eq. cost_function);
* adjoint L^dag_1 r = (1/T) r_s + u r_x - r_xx - r_xxxx and
  L^dag_2 = int int (1/T^2) u_s r dx ds (Sec. 4.1, Eq. KS_L_dagger; App. B);
* loop flow du/dtau = -L^dag_1, dT/dtau = -L^dag_2 (Eq. KS_G);
* discretisation: M x N Fourier modes on the uniform grid (m L / M, n / N), synthesis
  without a 1/N factor (Sec. 4.2, Eq. 2D_Fourier); derivatives in spectral space, products
  on the grid, 2/3-rule dealiasing in x and s (Sec. 4.2);
* tau-integration: IMEX Euler for u (the diagonal linear symbol Lambda_jk implicit, the
  remaining nonlinear part explicit) and explicit Euler for T, with the T integral taken as
  L x the (0,0) mode of the grid product (Sec. 4.2).  An EXPLICIT Euler variant is provided
  for small-step tests.

Readings where the paper is silent (each also listed in the design notes):

* Dealiasing placement: the state u is kept in the 2/3 band; each grid product (u u_x and
  u r_x) is transformed forward and truncated to the band, so r and L^dag_1 r are band
  limited.  The cut-off keeps |j| <= floor(M/3), |k| <= floor(N/3) and zeroes the Nyquist
  modes.
* The two-stage form r -> L^dag_1 r is the flow that is integrated (it is the exact
  gradient of the discrete J).  The expanded form G_1,L + G_1,NL of Eq. KS_G_1 is provided
  separately as an independent check (``flow_expanded``).
* IMEX: Lambda_jk uses T at the start of the step; u and T are both advanced from the same
  state l^n.
* Names: ``G`` is +L^dag_1 r (the ascent direction); ``dJdT`` is dJ/dT = 2 L^dag_2.
* Extrapolation (App. C): ``descend_extrapolated`` observes the loop every ``chunk`` steps and,
  from sqrt(J) <= 1e-3 on, each time sqrt(J) has halved since its anchor, moves it to
  l_b + (l_b - l_a) rho / (1 - rho), rho = sqrt(J_b) / sqrt(J_a), keeping the move only if it
  lowers sqrt(J) (the paper gives no formula; this geometric reading is exact for one decaying
  eigendirection, which is how it is pinned).
* Centre-symmetric subspace (Sec. 4.1, Eq. KS_loop_sym; Sec. 4.4): with ``xi=True`` the loop is
  restricted to the fields invariant under Xi: (x, s) -> (-x, s), u -> -u.  The input is
  projected onto that subspace with the band, and the descent direction L^dag_1 r is
  projected at every step (the flow preserves the symmetry of an invariant loop, so the
  projection only removes rounding; it also makes the returned G the gradient of J within
  the subspace).

The grid layout is u[n, m] (n: s-sample, m: x-sample).  Spectral arrays are indexed by
signed modes in the paper's ranges, k = -N/2 .. N/2-1 on axis 0 and j = -M/2 .. M/2-1 on
axis 1.
"""
from __future__ import annotations

import math

import numpy as np

EXPLICIT = 0
IMEX = 1


# ---------------------------------------------------------------------------------------
# Discretisation (Sec. 4.2, Eq. 2D_Fourier)
# ---------------------------------------------------------------------------------------

def signed_modes(M: int) -> np.ndarray:
    """Mode indices -M/2 .. M/2-1, the range of the paper's double sum (Eq. 2D_Fourier)."""
    return np.arange(-(M // 2), M - M // 2, dtype=np.int64)


def dft_matrix(M: int) -> np.ndarray:
    """E[m, j] = exp(2 pi i m j / M) for grid index m and signed mode j.

    The integer product m*j is reduced mod M before forming the angle so every entry is
    cos/sin of 2 pi t / M with 0 <= t < M, accurate to about one ulp.
    """
    m = np.arange(M, dtype=np.int64)[:, None]
    j = signed_modes(M)[None, :]
    t = np.mod(m * j, M).astype(np.float64)
    ang = 2.0 * math.pi * t / M
    return np.cos(ang) + 1j * np.sin(ang)


class Grid:
    """Dense DFT operators and wavenumbers for one (M, N, L) discretisation."""

    def __init__(self, Nx: int, Ns: int, L: float):
        self.Nx, self.Ns, self.L = int(Nx), int(Ns), float(L)
        self.Ex = dft_matrix(self.Nx)          # [m, j]
        self.Es = dft_matrix(self.Ns)          # [n, k]
        self.j = signed_modes(self.Nx)         # spatial modes (axis 1)
        self.k = signed_modes(self.Ns)         # temporal modes (axis 0)
        self.q = 2.0 * math.pi * self.j / self.L        # q_j = 2 pi j / L
        self.omega = 2.0 * math.pi * self.k             # omega_k = 2 pi k (s has period 1)
        self.Kx = self.Nx // 3
        self.Ks = self.Ns // 3
        # 2/3 rule in both directions (Sec. 4.2)
        self.mask = (np.abs(self.k)[:, None] <= self.Ks) & (np.abs(self.j)[None, :] <= self.Kx)
        self.Q = np.broadcast_to(self.q[None, :], (self.Ns, self.Nx))
        self.W = np.broadcast_to(self.omega[:, None], (self.Ns, self.Nx))

    # synthesis of Eq. 2D_Fourier: u(x_m, s_n) = sum_jk uh_jk exp(2 pi i (m j / M + n k / N))
    def to_grid(self, uh: np.ndarray) -> np.ndarray:
        return self.Es @ uh @ self.Ex.T

    # analysis, the inverse of to_grid: uh_jk = (1/(M N)) sum_mn u_mn exp(-2 pi i (...))
    def to_spectral(self, u: np.ndarray) -> np.ndarray:
        return (self.Es.conj().T @ u @ self.Ex.conj()) / (self.Nx * self.Ns)

    def project(self, uh: np.ndarray) -> np.ndarray:
        """P: zero every mode outside |j| <= floor(M/3), |k| <= floor(N/3)."""
        return np.where(self.mask, uh, 0.0)

    def xi(self, uh: np.ndarray) -> np.ndarray:
        """Spectral image of Xi u (x, s) = -u(-x, s) (Eq. KS_loop_sym): uh_jk -> -uh_{-j,k}.

        On the signed range j = -M/2 .. M/2-1 the mode -j sits at index (M - i) mod M of the
        mode at index i (the Nyquist mode maps to itself)."""
        neg = np.mod(self.Nx - np.arange(self.Nx), self.Nx)
        return -uh[:, neg]

    def xi_project(self, uh: np.ndarray) -> np.ndarray:
        """Orthogonal projection onto the Xi-invariant loops, (u + Xi u) / 2."""
        return 0.5 * (uh + self.xi(uh))

    def real_grid(self, uh: np.ndarray) -> np.ndarray:
        return self.to_grid(uh).real

    def dx(self, uh):
        return 1j * self.Q * uh

    def ds(self, uh):
        return 1j * self.W * uh


_GRIDS: dict = {}


def grid(Nx: int, Ns: int, L: float) -> Grid:
    key = (int(Nx), int(Ns), float(L))
    g = _GRIDS.get(key)
    if g is None:
        g = _GRIDS[key] = Grid(*key)
    return g


# ---------------------------------------------------------------------------------------
# Residual, cost and adjoint (Sec. 2, Sec. 4.1, App. B)
# ---------------------------------------------------------------------------------------

def band_state(u: np.ndarray, L: float, xi: bool = False) -> np.ndarray:
    """Project grid values onto the 2/3 band: uh = P F[u] (and onto the Xi subspace if xi)."""
    g = grid(u.shape[1], u.shape[0], L)
    uh = g.project(g.to_spectral(np.asarray(u, dtype=np.float64)))
    return g.xi_project(uh) if xi else uh


def residual_hat(uh: np.ndarray, T: float, g: Grid):
    """Spectral residual of Eq. KS_R with the u u_x product dealiased (Sec. 4.2).

    r_hat = -(1/T) (i omega) uh - P F[u u_x] - (i q)^2 uh - (i q)^4 uh.
    Returns (r_hat, u, u_x) with u, u_x on the grid.
    """
    u = g.real_grid(uh)
    ux = g.real_grid(g.dx(uh))
    nl = g.project(g.to_spectral(u * ux))
    uxx_h = (1j * g.Q) ** 2 * uh
    uxxxx_h = (1j * g.Q) ** 4 * uh
    rh = -(1.0 / T) * g.ds(uh) - nl - uxx_h - uxxxx_h
    return rh, u, ux


def cost(rh: np.ndarray, g: Grid) -> float:
    """J = int int r^2 dx ds (Eq. cost_function), as L x the grid mean of r^2.

    r is band limited, so r^2 has no aliased modes and the grid mean equals the integral
    over the unit s-period divided by L.
    """
    r = g.real_grid(rh)
    return float(g.L * np.mean(r * r))


def adjoint_T(uh: np.ndarray, rh: np.ndarray, T: float, g: Grid) -> float:
    """L^dag_2 = int int (1/T^2) u_s r dx ds (Eq. KS_L_dagger).

    Evaluated as the paper does for the period update (Sec. 4.2): the integrand is formed
    on the grid, transformed, and the (0,0) Fourier mode times L is the integral.
    """
    us = g.real_grid(g.ds(uh))
    r = g.real_grid(rh)
    prod_h = g.to_spectral(us * r / (T * T))
    i0 = g.Ns // 2  # index of k = 0 on axis 0
    j0 = g.Nx // 2  # index of j = 0 on axis 1
    return float(g.L * prod_h[i0, j0].real)


def adjoint_u_hat(uh: np.ndarray, rh: np.ndarray, T: float, g: Grid, u=None) -> np.ndarray:
    """Spectral L^dag_1 r = (1/T) r_s + u r_x - r_xx - r_xxxx (Eq. KS_L_dagger, App. B).

    The u r_x product is formed on the grid and truncated to the band (Sec. 4.2).
    """
    if u is None:
        u = g.real_grid(uh)
    rx = g.real_grid(g.dx(rh))
    nl = g.project(g.to_spectral(u * rx))
    rs_h = g.ds(rh)
    rxx_h = (1j * g.Q) ** 2 * rh
    rxxxx_h = (1j * g.Q) ** 4 * rh
    return (1.0 / T) * rs_h + nl - rxx_h - rxxxx_h


def residual(u: np.ndarray, T: float, L: float, xi: bool = False) -> dict:
    """Residual of the loop [P u; T] on the grid, with J and dJ/dT (Eq. KS_R, cost_function)."""
    g = grid(u.shape[1], u.shape[0], L)
    uh = band_state(u, L, xi)
    rh, _, _ = residual_hat(uh, T, g)
    J = cost(rh, g)
    L2 = adjoint_T(uh, rh, T, g)
    return {"uh": uh, "rh": rh, "r": g.real_grid(rh), "J": J, "L2": L2, "dJdT": 2.0 * L2}


def adjoint_grad(u: np.ndarray, T: float, L: float, xi: bool = False) -> dict:
    """G = +L^dag_1 r on the grid and dJ/dT = 2 L^dag_2, at the loop [P u; T].

    With xi, u is first projected onto the Xi subspace and G is the projected L^dag_1 r."""
    g = grid(u.shape[1], u.shape[0], L)
    uh = band_state(u, L, xi)
    rh, ug, _ = residual_hat(uh, T, g)
    Gh = adjoint_u_hat(uh, rh, T, g, u=ug)
    if xi:
        Gh = g.xi_project(Gh)
    L2 = adjoint_T(uh, rh, T, g)
    return {"uh": uh, "rh": rh, "Gh": Gh, "G": g.real_grid(Gh), "J": cost(rh, g),
            "L2": L2, "dJdT": 2.0 * L2}


# ---------------------------------------------------------------------------------------
# Linear symbol and tau-integration (Sec. 4.2)
# ---------------------------------------------------------------------------------------

def linear_symbol(T: float, g: Grid) -> np.ndarray:
    """Lambda_jk = -(2 pi k / T)^2 - q^8 + 2 q^6 - q^4, q = 2 pi j / L (Sec. 4.2)."""
    Q, W = g.Q, g.W
    return -(W / T) ** 2 - Q ** 8 + 2.0 * Q ** 6 - Q ** 4


def step_hat(uh: np.ndarray, T: float, g: Grid, dtau: float, scheme: int, xi: bool = False):
    """One tau-step of Eq. KS_G from the band state (uh, T).

    Returns (uh_next, T_next, J, L2) where J and L2 are evaluated at the input state.
    IMEX (Sec. 4.2): (uh' - uh)/dtau = Lambda uh' + G_NL with G_NL the field flow minus
    its linear part, G_NL = -L^dag_1 r - Lambda uh; explicit Euler for T.  With xi the field
    flow is the Xi-projected one (Lambda is even in j, so it commutes with the projection).
    """
    rh, u, _ = residual_hat(uh, T, g)
    J = cost(rh, g)
    L2 = adjoint_T(uh, rh, T, g)
    Gh = adjoint_u_hat(uh, rh, T, g, u=u)
    if xi:
        Gh = g.xi_project(Gh)
    flow = -Gh                      # du/dtau = -L^dag_1 (Eq. KS_G)
    if scheme == IMEX:
        lam = linear_symbol(T, g)
        g_nl = flow - lam * uh
        uh_next = g.project((uh + dtau * g_nl) / (1.0 - dtau * lam))
    elif scheme == EXPLICIT:
        uh_next = g.project(uh + dtau * flow)
    else:
        raise ValueError("scheme must be EXPLICIT (0) or IMEX (1)")
    T_next = T - dtau * L2          # dT/dtau = -L^dag_2, explicit Euler
    return uh_next, T_next, J, L2


def descend(u: np.ndarray, T: float, L: float, dtau: float, scheme: int, nsteps: int,
            tol: float = 0.0, record: bool = False, xi: bool = False) -> dict:
    """Advance the loop [P u; T] by up to ``nsteps`` tau-steps.

    Stops before a step whose starting state already has sqrt(J) < tol (the convergence
    test of Sec. 4.3).  Returns the final grid field, T, the step count, sqrt(J) of the final
    state and, optionally, the sqrt(J) history (one value per evaluated state).  With xi the
    descent runs in the Xi-invariant subspace (see ``step_hat``).
    """
    g = grid(u.shape[1], u.shape[0], L)
    uh = band_state(u, L, xi)
    hist = []
    steps = 0
    while True:
        rh, _, _ = residual_hat(uh, T, g)
        J = cost(rh, g)
        sq = math.sqrt(max(J, 0.0))
        if record:
            hist.append(sq)
        if (tol > 0.0 and sq < tol) or steps >= nsteps:
            break
        uh, T, _, _ = step_hat(uh, T, g, dtau, scheme, xi)
        steps += 1
    out = {"u": g.real_grid(uh), "uh": uh, "T": T, "steps": steps, "sqrtJ": sq}
    if record:
        out["hist"] = np.array(hist)
    return out


def sqrt_cost(uh: np.ndarray, T: float, g: Grid) -> float:
    """sqrt(J) of the band state (uh, T): the convergence measure of Sec. 4.3."""
    rh, _, _ = residual_hat(uh, T, g)
    return math.sqrt(max(cost(rh, g), 0.0))


def descend_extrapolated(u: np.ndarray, T: float, L: float, dtau: float, scheme: int,
                         nsteps: int, tol: float, chunk: int, start: float = 1e-3,
                         drop: float = 0.5, xi: bool = False) -> dict:
    """Tau-descent accelerated by linear extrapolation along the trajectory (App. C).

    App. C alternates integration of Eq. KS_G with an extrapolation along the leading
    eigendirection of the linearised loop dynamics about the attracting loop: the first one
    once sqrt(J) has reached ``start`` (1e-3 in its example), and then each time sqrt(J) has
    halved since the previous one (``drop`` = 1/2).  The paper gives no formula; the reading
    used here: the loop is observed every ``chunk`` steps; below ``start`` the first
    observation becomes the anchor l_a; at an observation l_b with sqrt(J_b) <= drop *
    sqrt(J_a), if the approach were a single decaying eigendirection, l(tau) = l* + c rho^tau,
    the fixed point would be l* = l_b + (l_b - l_a) rho / (1 - rho) with rho = sqrt(J_b) /
    sqrt(J_a) (J is quadratic in the distance to l*).  This l* (for the band state and T) is
    kept only if its sqrt(J) is below sqrt(J_b); either way the state the descent continues
    from becomes the next anchor.  The convergence test is that of ``descend``: stop before a
    step whose starting state has sqrt(J) < tol.

    Returns the final grid field, T, the step count, sqrt(J) of the final state, and the
    numbers of extrapolations kept and rejected.
    """
    g = grid(u.shape[1], u.shape[0], L)
    uh = band_state(u, L, xi)
    steps = 0
    anchor = None            # (uh, T, sqrt(J)) at the start of the current halving segment
    kept = rejected = 0
    converged = False
    while steps < nsteps and not converged:
        for _ in range(min(chunk, nsteps - steps)):
            if sqrt_cost(uh, T, g) < tol:
                converged = True
                break
            uh, T, _, _ = step_hat(uh, T, g, dtau, scheme, xi)
            steps += 1
        if converged:
            break
        sq = sqrt_cost(uh, T, g)
        if not sq <= start:
            continue
        if anchor is None:
            anchor = (uh, T, sq)
            continue
        if sq > drop * anchor[2]:
            continue
        rho = sq / anchor[2]
        c = rho / (1.0 - rho)
        uh_e = uh + (uh - anchor[0]) * c
        T_e = T + (T - anchor[1]) * c
        sq_e = sqrt_cost(uh_e, T_e, g)
        if sq_e < sq:
            uh, T, sq = uh_e, T_e, sq_e
            kept += 1
        else:
            rejected += 1
        anchor = (uh, T, sq)
    return {"u": g.real_grid(uh), "uh": uh, "T": T, "steps": steps,
            "sqrtJ": sqrt_cost(uh, T, g), "extrapolations": kept, "rejected": rejected}


# ---------------------------------------------------------------------------------------
# Independent forms used only to pin the above (App. B; Eq. KS_G_1)
# ---------------------------------------------------------------------------------------

def directional_derivative(u: np.ndarray, T: float, v: np.ndarray, v2: float, L: float):
    """Field part of the directional derivative of the residual along [v; v2] (App. B):

        (v2 / T^2) u_s - (1/T) v_s - (u v)_x - v_xx - v_xxxx,

    with the product u v formed on the grid and truncated to the band.  Returns grid values.
    """
    g = grid(u.shape[1], u.shape[0], L)
    uh = band_state(u, L)
    vh = band_state(v, L)
    ug = g.real_grid(uh)
    vg = g.real_grid(vh)
    uvh = g.project(g.to_spectral(ug * vg))
    out_h = ((v2 / (T * T)) * g.ds(uh) - (1.0 / T) * g.ds(vh) - g.dx(uvh)
             - (1j * g.Q) ** 2 * vh - (1j * g.Q) ** 4 * vh)
    return g.real_grid(out_h)


def adjoint_operator(u: np.ndarray, T: float, w: np.ndarray, L: float):
    """Generalized-loop adjoint applied to [w; 0] (App. B): returns (field part on the grid,
    scalar part) = ((1/T) w_s + u w_x - w_xx - w_xxxx, int int (1/T^2) u_s w)."""
    g = grid(u.shape[1], u.shape[0], L)
    uh = band_state(u, L)
    wh = band_state(w, L)
    f_h = adjoint_u_hat(uh, wh, T, g)
    return g.real_grid(f_h), adjoint_T(uh, wh, T, g)


def flow_expanded(u: np.ndarray, T: float, L: float) -> np.ndarray:
    """du/dtau written out in u alone, G_1,L + G_1,NL of Eq. KS_G_1 (Sec. 4.2).

    Every derivative is spectral; every product is formed on the grid and the sum is
    truncated to the band once.  For loops whose band is narrow enough that the cubic
    products do not alias, this equals -L^dag_1 r from the two-stage evaluation.
    """
    g = grid(u.shape[1], u.shape[0], L)
    uh = band_state(u, L)
    D = lambda a, b: g.real_grid((1j * g.Q) ** a * (1j * g.W) ** b * uh)  # noqa: E731
    u0 = D(0, 0)
    ux, uxx, uxxx, uxxxx = D(1, 0), D(2, 0), D(3, 0), D(4, 0)
    us, uss, uxs = D(0, 1), D(0, 2), D(1, 1)
    lin_h = ((1j * g.W) ** 2 / (T * T) - (1j * g.Q) ** 8 - 2.0 * (1j * g.Q) ** 6
             - (1j * g.Q) ** 4) * uh
    nl = (-5.0 * uxxxx * ux - 10.0 * uxxx * uxx - 3.0 * uxx * ux + u0 * u0 * uxx
          + u0 * ux * ux + (2.0 / T) * u0 * uxs + (1.0 / T) * ux * us)
    return g.real_grid(lin_h + g.project(g.to_spectral(nl)))


# ---------------------------------------------------------------------------------------
# Batched helpers (a batch is a list of independent loops)
# ---------------------------------------------------------------------------------------

def residual_batch(us, Ts, L, xi=False):
    return [residual(u, T, L, xi) for u, T in zip(us, Ts)]


def adjoint_grad_batch(us, Ts, L, xi=False):
    return [adjoint_grad(u, T, L, xi) for u, T in zip(us, Ts)]


def descend_batch(us, Ts, L, dtau, scheme, nsteps, tol=0.0, xi=False):
    return [descend(u, T, L, dtau, scheme, nsteps, tol, xi=xi) for u, T in zip(us, Ts)]


# ---------------------------------------------------------------------------------------
# Time integration of the KSE itself, for the initial guesses (Sec. 4.3)
# ---------------------------------------------------------------------------------------
# The paper takes its initial loops from a chaotic solution u(x, t) of u_t = -u u_x - u_xx
# - u_xxxx on [0, L) (Sec. 4.3); it does not name the integrator.  Reading: a Fourier
# pseudo-spectral discretisation with Nx points, 2/3-rule dealiasing of the product (as in the
# descent, Sec. 4.2), and fourth-order exponential time differencing (ETDRK4 of Cox & Matthews,
# J. Comput. Phys. 176, 2002), whose linear part is the exact diagonal symbol q^2 - q^4.  Here
# everything is a dense DFT over the signed modes, and the phi-functions come from their power
# series or closed forms (not a contour integral).  parity pins: a conserved mean, a constant
# state, fourth-order convergence under dt halving, agreement with classical RK4 at a step far
# inside its stability limit, and the centre-symmetric subspace kept exactly.

def etd_phi(z: np.ndarray):
    """phi_1, phi_2, phi_3 at real z: phi_k(z) = sum_{m >= 0} z^m / (m + k)!.

    |z| < 1: the series (30 terms); otherwise phi_1 = (e^z - 1) / z, phi_2 = (phi_1 - 1) / z,
    phi_3 = (phi_2 - 1/2) / z."""
    z = np.asarray(z, dtype=np.float64)
    p1 = np.empty_like(z)
    p2 = np.empty_like(z)
    p3 = np.empty_like(z)
    small = np.abs(z) < 1.0
    zs = z[small]
    s1 = np.zeros_like(zs)
    s2 = np.zeros_like(zs)
    s3 = np.zeros_like(zs)
    for m in range(29, -1, -1):                      # Horner from the smallest term
        s1 = s1 * zs + 1.0 / math.factorial(m + 1)
        s2 = s2 * zs + 1.0 / math.factorial(m + 2)
        s3 = s3 * zs + 1.0 / math.factorial(m + 3)
    p1[small], p2[small], p3[small] = s1, s2, s3
    zl = z[~small]
    q1 = np.expm1(zl) / zl
    q2 = (q1 - 1.0) / zl
    q3 = (q2 - 0.5) / zl
    p1[~small], p2[~small], p3[~small] = q1, q2, q3
    return p1, p2, p3


def dns_coefficients(L: float, Nx: int, dt: float):
    """Wavenumbers, dealiasing mask, and the ETDRK4 weights of each signed x-mode j:
    E = e^z, E2 = e^(z/2), Q = (dt/2) phi_1(z/2), f1 = dt (phi_1 - 3 phi_2 + 4 phi_3)(z),
    f2 = dt (phi_2 - 2 phi_3)(z), f3 = dt (4 phi_3 - phi_2)(z), with z = dt (q_j^2 - q_j^4)."""
    j = signed_modes(Nx)
    q = 2.0 * math.pi * j / L
    keep = (np.abs(j) <= Nx // 3) & (np.abs(j) != Nx // 2)
    z = dt * (q ** 2 - q ** 4)
    a1, a2, a3 = etd_phi(z)
    h1, _, _ = etd_phi(z / 2.0)
    return dict(q=q, keep=keep, E=np.exp(z), E2=np.exp(z / 2.0), Q=0.5 * dt * h1,
                f1=dt * (a1 - 3.0 * a2 + 4.0 * a3), f2=dt * (a2 - 2.0 * a3),
                f3=dt * (4.0 * a3 - a2))


def dns_nonlinear(vh: np.ndarray, q: np.ndarray, keep: np.ndarray, Ex: np.ndarray) -> np.ndarray:
    """-(u u_x) = -(u^2 / 2)_x in spectral space, product on the grid, truncated to the 2/3 band.
    vh: coefficients over the signed modes with u(x_m) = (1/Nx) sum_j vh_j e^(i q_j x_m)."""
    Nx = vh.shape[0]
    u = np.real(Ex @ vh) / Nx
    W = Ex.conj().T @ (u * u)
    return np.where(keep, -0.5j * q * W, 0.0)


def dns(L: float, Nx: int, dt: float, nsteps: int, u0: np.ndarray, save_every: int = 1,
        symmetric: bool = False):
    """ETDRK4 integration of the KSE from the grid field u0 [Nx]; returns (t [nsave],
    u [nsave, Nx]) every save_every steps, t = 0 first.  symmetric: the state is kept in the
    centre-symmetric subspace u(-x) = -u(x) (purely imaginary coefficients), projected
    initially and after every step."""
    c = dns_coefficients(L, Nx, dt)
    Ex = dft_matrix(Nx)
    q, keep = c["q"], c["keep"]
    sym = (lambda v: 1j * v.imag) if symmetric else (lambda v: v)  # noqa: E731
    N = lambda v: dns_nonlinear(v, q, keep, Ex)  # noqa: E731
    vh = sym(np.where(keep, Ex.conj().T @ np.asarray(u0, dtype=np.float64), 0.0))
    ts, us = [0.0], [np.real(Ex @ vh) / Nx]
    for n in range(1, nsteps + 1):
        Nv = N(vh)
        a = c["E2"] * vh + c["Q"] * Nv
        Na = N(a)
        b = c["E2"] * vh + c["Q"] * Na
        Nb = N(b)
        cc = c["E2"] * a + c["Q"] * (2.0 * Nb - Nv)
        Nc = N(cc)
        vh = sym(c["E"] * vh + c["f1"] * Nv + 2.0 * c["f2"] * (Na + Nb) + c["f3"] * Nc)
        if n % save_every == 0:
            ts.append(n * dt)
            us.append(np.real(Ex @ vh) / Nx)
    return np.asarray(ts), np.asarray(us)


def dns_rk4(L: float, Nx: int, dt: float, nsteps: int, u0: np.ndarray) -> np.ndarray:
    """Classical RK4 on the same dealiased Fourier system (v' = (q^2 - q^4) v + N(v)); an
    independent integrator for pinning ``dns`` (stable only for dt below ~2.8 / max q^4)."""
    j = signed_modes(Nx)
    q = 2.0 * math.pi * j / L
    keep = (np.abs(j) <= Nx // 3) & (np.abs(j) != Nx // 2)
    lam = q ** 2 - q ** 4
    Ex = dft_matrix(Nx)
    f = lambda v: np.where(keep, lam * v, 0.0) + dns_nonlinear(v, q, keep, Ex)  # noqa: E731
    vh = np.where(keep, Ex.conj().T @ np.asarray(u0, dtype=np.float64), 0.0)
    for _ in range(nsteps):
        k1 = f(vh)
        k2 = f(vh + 0.5 * dt * k1)
        k3 = f(vh + 0.5 * dt * k2)
        k4 = f(vh + dt * k3)
        vh = vh + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    return np.real(Ex @ vh) / Nx


def norm_series(us: np.ndarray, L: float) -> np.ndarray:
    """||u||(t) = (int_0^L u^2 dx)^(1/2) of each saved field u[i, m] (Sec. 4.3), the grid mean
    of u^2 times L (exact for the dealiased fields of the run: u^2 has no aliased modes)."""
    us = np.asarray(us, dtype=np.float64)
    return np.sqrt(L * np.mean(us * us, axis=-1))


def segment_loop(ts: np.ndarray, us: np.ndarray, a: int, T: float, Ns: int) -> np.ndarray:
    """The field of a recurrence loop (Sec. 4.3) before its low-pass: the saved run u(x_m, t_i)
    at the Ns instants t_a + T n / Ns, n = 0..Ns-1, by linear interpolation in time between the
    saved instants (np.interp per grid point).  Returns [Ns, Nx]."""
    us = np.asarray(us, dtype=np.float64)
    s_t = ts[a] + T * np.arange(Ns) / Ns
    return np.stack([np.interp(s_t, ts, us[:, m]) for m in range(us.shape[1])], axis=1)
