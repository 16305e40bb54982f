"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: numerical
quadrature of the Hankel transform (Eq. (11)), closed forms of the
band-limited Gaussian, Poisson summation, DFT inversion at lattice points,
exact translation identities, brute force on tiny inputs, and the far-field
error bound of the scaled Lemma (Eq. (33)).
"""
import itertools
import os

import numpy as np
import pytest
from scipy import integrate, special

import oracle as O


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


# ---------------------------------------------------------------- T-FT ----
@pytest.mark.parametrize("d", [1, 2, 3, 5])
def test_gaussian_ft_matches_hankel_quadrature(d):
    """Eq. (11) by quadrature vs the oracle's closed-form Gaussian transform.

    The oracle's closed-form coefficients are C = (2pi)^-d Phi_hat with
    Phi_hat(xi) = (pi/eps^2)^{d/2} exp(-|xi|^2/(4 eps^2)) (Eq. (5) convention);
    the table of transforms (Sec. 3) prints the same function times (2pi)^{-d/2}."""
    eps, M, L = 1.5, 8, 3.0
    wc = O.coeffs_closed_gaussian(eps, d, M, L)
    xi, w = O.freq_grid(M, L)
    # one-dimensional cut through the grid along dimension 0, others at xi=0
    mid = M // 2
    idx = [mid + (M + 1) * 0] * 1
    for kk in range(M + 1):
        m = kk + sum(mid * (M + 1) ** t for t in range(1, d))
        wprod = w[kk] * w[mid] ** (d - 1)
        phi_hat = wc[m] / wprod * (2 * np.pi) ** d
        r = abs(xi[kk])
        nu = (d - 2) / 2.0
        if r == 0.0:
            # limit r -> 0 of Eq. (11): surface area form
            ref = (2 * np.pi) ** (d / 2) * integrate.quad(
                lambda t: np.exp(-(eps * t) ** 2) * t ** (d - 1) / (2 ** nu * special.gamma(nu + 1)),
                0, np.inf)[0]
        else:
            ref = (2 * np.pi) ** (d / 2) * r ** (-nu) * integrate.quad(
                lambda t: np.exp(-(eps * t) ** 2) * t ** (d / 2) * special.jv(nu, r * t),
                0, 12.0 / eps, limit=400)[0]
        table = np.exp(-(r / eps) ** 2 / 4) / np.sqrt(2) ** d / eps ** d * (2 * np.pi) ** (d / 2)
        assert abs(phi_hat - ref) <= 1e-10 * max(1.0, abs(ref))
        assert abs(phi_hat - table) <= 1e-12 * max(1.0, abs(table))
    assert idx  # silence linters


@pytest.mark.parametrize("d", [1, 3, 5])
def test_imq_table_row_matches_hankel(d):
    """The table's IMQ row sqrt(2/pi) K_nu(|xi|)/|xi|^nu, nu=(d-1)/2, times (2pi)^{d/2},
    is Eq. (11) of 1/sqrt(1+t^2).  Pins the (2pi)^{-d/2} normalisation reading
    that the coefficient formula corrects for."""
    nu = (d - 1) / 2.0
    for r in (0.7, 1.9, 4.0):
        table = (2 * np.pi) ** (d / 2) * np.sqrt(2 / np.pi) * special.kv(nu, r) / r ** nu
        # Eq. (11) with J_{(d-2)/2}; oscillatory tail handled by quad's Fourier weight
        # via the closed forms of J for half-integer order (d odd).
        if d == 1:
            val = 2 * integrate.quad(lambda t: 1 / np.sqrt(1 + t * t), 0, np.inf, weight="cos", wvar=r)[0]
        elif d == 3:
            val = 4 * np.pi / r * integrate.quad(lambda t: t / np.sqrt(1 + t * t), 0, np.inf,
                                                 weight="sin", wvar=r)[0]
        else:  # d == 5: J_{3/2}(z) = sqrt(2/(pi z)) (sin z / z - cos z)
            c = (2 * np.pi) ** 2.5 * r ** -1.5 * np.sqrt(2 / (np.pi * r))
            s1 = integrate.quad(lambda t: t / np.sqrt(1 + t * t) / r, 0, np.inf, weight="sin", wvar=r)[0]
            s2 = integrate.quad(lambda t: t * t / np.sqrt(1 + t * t) - t, 0, np.inf, weight="cos", wvar=r)[0]
            s2 += -1.0 / r ** 2  # int_0^inf t cos(rt) dt in the Abel sense
            val = c * (s1 - s2)
        assert abs(val - table) <= 2e-6 * abs(table)


# ------------------------------------------------------------- T-BL ------
def _bl_gauss_1d(t, eps, sigma):
    """(1/2pi) int_{-sigma}^{sigma} phi_hat(xi) e^{i xi t} dxi for phi = exp(-(eps t)^2),
    closed form exp(-(eps t)^2) Re erf(sigma/(2 eps) + i eps t), evaluated through
    the Faddeeva function to avoid overflow."""
    a = sigma / (2 * eps)
    b = eps * np.asarray(t, dtype=np.float64)
    val = np.exp(-b * b) - np.exp(-a * a) * np.exp(-2j * a * b) * special.wofz(-b + 1j * a)
    return val.real


def test_bandlimited_gaussian_closed_form_and_bound():
    """Sec. 3.2's band-limited integral, closed form vs quadrature, and the
    band-limit error |Phi_sigma - Phi| <= erfc(sigma/(2 eps))."""
    eps, sigma = 4.0, 20.0
    ts = np.linspace(-1.2, 1.2, 41)
    for t in ts[::5]:
        q = integrate.quad(lambda x: np.sqrt(np.pi) / eps * np.exp(-x * x / (4 * eps * eps)) * np.cos(x * t),
                           -sigma, sigma, limit=200)[0] / (2 * np.pi)
        assert abs(_bl_gauss_1d(t, eps, sigma) - q) < 1e-13
    err = np.max(np.abs(_bl_gauss_1d(ts, eps, sigma) - np.exp(-(eps * ts) ** 2)))
    # the bound is attained at t = 0, where Phi_sigma(0) = erf(sigma/(2 eps))
    assert err <= special.erfc(sigma / (2 * eps)) * (1 + 1e-12)
    assert err > 0.999 * special.erfc(sigma / (2 * eps))


# -------------------------------------------------------------- T-Q ------
@pytest.mark.parametrize("d", [1, 2])
def test_poisson_closed_form_coefficients(d):
    """With closed-form C, K(r) = prod_t sum_n Phi_sigma(r_t + nL) (Poisson summation),
    where Phi_sigma is the band-limited Gaussian.  The band edge is kept large
    (exp(-sigma^2/(4eps^2)) ~ 1e-4) so the half weights at +-sigma matter."""
    eps, M, L = 4.0, 16, 2.5
    sigma = np.pi * M / L
    wc = O.coeffs_closed_gaussian(eps, d, M, L)
    rng = np.random.default_rng(5)
    r = rng.uniform(-1.0, 1.0, (12, d))
    K = O.kernel_K(wc, d, M, L, r)
    # the image sum converges like 1/n (sinc tail of Phi_sigma): symmetric partial
    # sums S_N, S_2N and one Richardson step 2 S_2N - S_N remove the 1/N term
    def image_sum(x, nmax):
        n = np.arange(-nmax, nmax + 1)
        return np.sum(_bl_gauss_1d(x + n * L, eps, sigma))
    ref = np.ones(len(r))
    for t in range(d):
        ref *= np.array([2 * image_sum(x, 200000) - image_sum(x, 100000) for x in r[:, t]])
    assert np.max(np.abs(K - ref)) < 1e-12
    assert np.max(np.abs(K - np.exp(-eps ** 2 * np.sum(r * r, axis=1)))) > 1e-5  # band edge visible


# ------------------------------------------------------------ T-SAMP -----
@pytest.mark.parametrize("kernel,eps,d,M,L,alpha", [(O.IMQ, 2.0, 2, 16, 4.0, 4.5),
                                                    (O.IMQ, 2.0, 3, 12, 4.0, 4.5),
                                                    (O.GAUSSIAN, 3.0, 3, 10, 3.0, 0.0),
                                                    (O.MQ, 2.0, 2, 16, 4.0, 4.5),
                                                    (O.WENDLAND, 0.5, 2, 16, 4.0, 0.0)])
def test_sampled_coefficients_interpolate_lattice(kernel, eps, d, M, L, alpha):
    """DFT inversion: with sampled C, K(qh) equals the periodised, windowed sample f(q)
    exactly, and f(q) is Phi(qh) inside the window's flat part."""
    wc = O.coeffs_sampled(kernel, eps, d, M, L, alpha, 1.0)
    f = O.lattice_samples(kernel, eps, d, M, L, alpha, 1.0)
    h = L / M
    qs = np.array(list(itertools.product(range(-M // 2, M // 2), repeat=d)))
    rng = np.random.default_rng(2)
    pick = qs[rng.choice(len(qs), size=min(200, len(qs)), replace=False)]
    K = O.kernel_K(wc, d, M, L, pick * h)
    fv = f[tuple((pick + M // 2).T)]
    assert np.max(np.abs(K - fv)) < 1e-13 * max(1.0, np.max(np.abs(fv)))
    inner = np.max(np.abs(pick * h), axis=1) <= 1.0
    phi_v = O.phi(kernel, eps, np.linalg.norm(pick[inner] * h, axis=1))
    assert np.max(np.abs(fv[inner] - phi_v)) < 2e-9


def test_sampled_matches_closed_form_gaussian():
    """For the Gaussian with negligible images, the sampled coefficients are the
    closed-form Fourier transform up to aliasing (Eq. (M2Loperator) vs Eq. (29))."""
    eps, d, M, L = 3.0, 2, 32, 3.0
    a = O.coeffs_sampled(O.GAUSSIAN, eps, d, M, L, 0.0, 1.0)
    b = O.coeffs_closed_gaussian(eps, d, M, L)
    assert np.max(np.abs(a - b)) < 1e-10 * np.max(np.abs(b))


# ------------------------------------------------------------ T-TREE -----
def _tree_case(d, N, D, seed):
    rng = np.random.default_rng(seed)
    X = rng.random((N, d))
    # points on faces, edges and the far corner exercise floor + clamp
    X[0] = 1.0
    X[1] = 0.5
    X[2, 0] = 0.0
    X[3] = 0.25
    return X


def test_morton_keys_by_hand():
    """Keys from the definition, worked by hand (d=2, D=2, dimension 0 in bit 0):
    (0.3, 0.8) -> k=(1,3) -> bits (k0b0,k1b0,k0b1,k1b1)=(1,1,0,1) -> 11;
    (1.0, 0.0) -> k=(3,0) (clamped) -> (1,0,1,0) -> 5;  (0.5, 0.5) -> k=(2,2) -> 12."""
    X = np.array([[0.3, 0.8], [1.0, 0.0], [0.5, 0.5]])
    T = O.tree(X, np.zeros(2), 1.0, 2)
    assert sorted(T["keys"].tolist()) == [5, 11, 12]
    assert T["perm"].tolist() == [1, 0, 2]


@pytest.mark.parametrize("d,N,D", [(2, 300, 3), (3, 400, 3), (2, 200, 4)])
def test_lists_cover_every_pair_once(d, N, D):
    """Every ordered pair (i, j) is either near (leaf Chebyshev distance <= 1) or in
    exactly one interaction list IL_l, l = 2..D; lists match brute-force definitions."""
    X = _tree_case(d, N, D, seed=d * 10 + D)
    T = O.tree(X, np.zeros(d), 1.0, D)
    # brute-force box coordinates of every point at every level, by repeated halving
    kD = np.empty((N, d), dtype=np.int64)
    for i in range(N):
        for t in range(d):
            kD[i, t] = min(max(int(np.floor(X[i, t] * 2 ** D)), 0), 2 ** D - 1)
    leaf_of_orig = np.searchsorted(T["leaf_key"], O.morton_encode(kD, d, D))
    count = np.zeros((N, N), dtype=np.int64)
    near_sets = [set(T["near_idx"][T["near_off"][a]:T["near_off"][a + 1]].tolist())
                 for a in range(len(T["leaf_key"]))]
    for i in range(N):
        for j in range(N):
            cheb = np.max(np.abs(kD[i] - kD[j]))
            is_near = leaf_of_orig[j] in near_sets[leaf_of_orig[i]]
            assert is_near == (cheb <= 1)
            count[i, j] += is_near
    for l in range(2, D + 1):
        lv = T["levels"][l]
        kl = kD >> (D - l)
        box = np.searchsorted(lv["key"], O.morton_encode(kl, d, l))
        ils = [set(lv["il_idx"][lv["il_off"][a]:lv["il_off"][a + 1]].tolist())
               for a in range(len(lv["key"]))]
        for i in range(N):
            for j in range(N):
                inil = box[j] in ils[box[i]]
                parent_near = np.max(np.abs((kl[i] >> 1) - (kl[j] >> 1))) <= 1
                far = np.max(np.abs(kl[i] - kl[j])) >= 2
                assert inil == (parent_near and far)
                count[i, j] += inil
    assert np.all(count == 1)
    # sizes: |N_a| <= 3^d, |IL| <= 6^d - 3^d
    assert np.max(np.diff(T["near_off"])) <= 3 ** d
    for l in range(2, D + 1):
        assert np.max(np.diff(T["levels"][l]["il_off"])) <= 6 ** d - 3 ** d


# ------------------------------------------------------------ T-CONS -----
def test_translation_consistency():
    """M2M(P2M(children)) = P2M at the parent and L2P(L2L(L_p)) = L2P of L_p at the
    parent: exact on one shared grid (Eqs. (43), (48) with P = I)."""
    d, D, M, L = 2, 3, 12, 3.0
    rng = np.random.default_rng(7)
    X = rng.random((300, d))
    lam = rng.standard_normal(300)
    T = O.tree(X, np.zeros(d), 1.0, D)
    ls = lam[T["perm"]]
    V3 = O.p2m(T, ls, M, L)
    V2 = O.m2m(T, V3, 3, M, L)
    # P2M straight at level 2: points grouped by their level-2 box
    lv2 = T["levels"][2]
    leaf_par = T["levels"][3]["parent"]
    off2 = np.searchsorted(T["leaf_off"][:-1], T["leaf_off"][:-1])  # identity, for clarity
    pt_off2 = np.array([T["leaf_off"][np.searchsorted(leaf_par, b)] for b in range(len(lv2["key"]))]
                       + [T["N"]])
    T2 = dict(T, leaf_key=lv2["key"], leaf_off=pt_off2, D=2)
    V2_direct = O.p2m(T2, ls, M, L)
    assert off2 is not None
    assert rel(V2, V2_direct) < 1e-13
    # L2P(L2L(Lp)) vs L2P of Lp at the parent level
    Lp = rng.standard_normal(V2.shape) + 1j * rng.standard_normal(V2.shape)
    Lc = np.zeros_like(V3)
    O.l2l(T, Lp, Lc, 3, M, L)
    u_child = np.zeros(T["N"])
    O.l2p(T, Lc, M, L, u_child)
    u_par = np.zeros(T["N"])
    O.l2p(T2, Lp, M, L, u_par)
    assert rel(u_child, u_par) < 1e-13


# ----------------------------------------------------------- T-BRUTE -----
@pytest.mark.parametrize("d,N,D,kernel,eps,M,L,alpha", [
    (2, 400, 3, O.GAUSSIAN, 4.0, 24, 2.5, 0.0),
    (2, 300, 4, O.IMQ, 2.0, 16, 4.0, 4.5),
    (3, 250, 3, O.IMQ, 2.0, 10, 4.0, 4.5),
    (3, 200, 2, O.GAUSSIAN, 3.0, 12, 3.0, 0.0),
    (2, 300, 3, O.MQ, 2.0, 16, 4.0, 4.5),
    (2, 300, 3, O.WENDLAND, 0.5, 16, 4.0, 0.0),
])
def test_fmm_equals_bruteforce(d, N, D, kernel, eps, M, L, alpha):
    """The multilevel FMM (P2M, M2M, M2L over IL_l, L2L, L2P) equals the direct sum of
    Phi over near pairs and K over all other pairs, computed pair by pair."""
    rng = np.random.default_rng(N + d)
    X = rng.random((N, d))
    lam = rng.standard_normal(N)
    T = O.tree(X, np.zeros(d), 1.0, D)
    wc = O.coeffs_sampled(kernel, eps, d, M, L, alpha, 1.0)
    u = O.fmm(T, lam, kernel, eps, wc, M, L)
    ub = O.fmm_brute(T, lam, kernel, eps, wc, M, L)
    assert rel(u, ub) < 1e-13
    ut = O.fmm_at_targets(T, lam, kernel, eps, wc, M, L, np.arange(0, N, 5))
    assert rel(ut, u[::5]) < 1e-13


# ------------------------------------------------------------- T-ERR -----
def test_fmm_error_within_lemma_bound_config1():
    """d=2, N=4096, Gaussian eps=4, depth 3: |u_fmm - u_direct|_i is bounded by
    max_far |K - Phi| * sum_j |lambda_j| (scaled Lemma, Eq. (33)); the actual
    relative L2 error is small."""
    from workloads import config1
    X, lam, p = config1()
    T = O.tree(X, np.zeros(2), 1.0, p["depth"])
    wc = O.coeffs_sampled(O.GAUSSIAN, p["eps"], 2, p["M"], p["L"], p["alpha"], 1.0)
    u = O.fmm(T, lam, O.GAUSSIAN, p["eps"], wc, p["M"], p["L"])
    ud = O.direct(X, lam, O.GAUSSIAN, p["eps"])
    rng = np.random.default_rng(11)
    r = rng.uniform(-1, 1, (4000, 2))
    r = r[np.max(np.abs(r), axis=1) >= 1.0 / 8]
    kerr = np.max(np.abs(O.kernel_K(wc, 2, p["M"], p["L"], r) - O.phi(O.GAUSSIAN, p["eps"],
                                                                       np.linalg.norm(r, axis=1))))
    bound = kerr * np.sum(np.abs(lam))
    assert np.max(np.abs(u - ud)) <= bound
    assert rel(u, ud) < 1e-10


# ------------------------------------------------------- direct sum ------
def test_direct_sum_small_cases():
    """Eq. (1) on two points, and the Gershgorin bound gamma_max <= N max|Phi|."""
    X = np.array([[0.0, 0.0], [0.3, 0.4]])
    lam = np.array([2.0, -1.0])
    u = O.direct(X, lam, O.GAUSSIAN, 2.0)
    g = np.exp(-(2.0 * 0.5) ** 2)
    assert np.allclose(u, [2.0 - g, 2.0 * g - 1.0], rtol=0, atol=1e-15)
    u = O.direct(X, lam, O.IMQ, 2.0)
    q = 1 / np.sqrt(1 + 1.0)
    assert np.allclose(u, [2.0 - q, 2.0 * q - 1.0], rtol=0, atol=1e-15)
    u = O.direct(X, lam, O.MQ, 2.0)
    m = np.sqrt(2.0)
    assert np.allclose(u, [2.0 - m, 2.0 * m - 1.0], rtol=0, atol=1e-15)
    u = O.direct(X, lam, O.WENDLAND, 0.5)          # eps r = 0.25: 0.75^3 * 1.75
    w = 0.73828125
    assert np.allclose(u, [2.0 - w, 2.0 * w - 1.0], rtol=0, atol=1e-15)
    u = O.direct(X, lam, O.WENDLAND, 2.0)          # eps r = 1: the support edge
    assert np.allclose(u, [2.0, -1.0], rtol=0, atol=1e-15)
    rng = np.random.default_rng(3)
    Y = rng.random((60, 3))
    A = np.stack([O.direct(Y, e, O.IMQ, 2.0) for e in np.eye(60)], axis=1)
    assert np.allclose(A, A.T, atol=1e-15)
    assert np.max(np.linalg.eigvalsh(A)) <= 60 * 1.0


def test_mq_matrix_has_one_positive_eigenvalue():
    """The multiquadric is conditionally negative definite of order 1 with
    Phi(0) > 0: its interpolation matrix on distinct centres has exactly one
    positive eigenvalue (Micchelli), which an IMQ or sign slip would break."""
    rng = np.random.default_rng(4)
    Y = rng.random((80, 2))
    A = np.stack([O.direct(Y, e, O.MQ, 3.0) for e in np.eye(80)], axis=1)
    ev = np.linalg.eigvalsh(A)
    assert np.sum(ev > 0) == 1 and np.all(ev[:-1] < 0)


# ----------------------------------------------------------- T-GMRES -----
def test_oracle_gmres_matches_dense_solve():
    """GMRES(m) with restarts reaches the dense LAPACK solution of a symmetric positive
    definite RBF system (IMQ eps=50, 300 centres), and the iteration stops at the tolerance."""
    from oracle.solver import gmres
    rng = np.random.default_rng(12)
    X = rng.random((300, 2))
    r = np.linalg.norm(X[:, None, :] - X[None, :, :], axis=2)
    A = O.phi(O.IMQ, 50.0, r)          # condition number ~3e3
    b = rng.standard_normal(300)
    x_ref = np.linalg.solve(A, b)
    x, it, hist = gmres(lambda v: A @ v, b, m=20, tol=1e-12, maxit=5000)
    assert np.linalg.norm(A @ x - b) <= 1e-12 * np.linalg.norm(b) * 1.01
    assert np.linalg.norm(x - x_ref) <= 1e-8 * np.linalg.norm(x_ref)
    assert len(hist) >= 2 and it > 20          # several restarts were exercised
    # gamma_max <= N max|Phi| (Gershgorin, Sec. 3.1)
    assert np.max(np.linalg.eigvalsh(A)) <= 300 * 1.0


# ---------------------------------------------- learned preconditioner ----
def test_oracle_mlp_gradient_matches_finite_differences():
    """T-MLP-FD: the oracle's backward pass equals central differences of the loss."""
    from oracle.solver import mlp_init, mlp_forward, mlp_backward, mse_loss
    rng = np.random.default_rng(6)
    W, b = mlp_init([12, 16, 16, 16, 5], seed=1)
    for bl in b:
        bl += 0.1 * rng.standard_normal(bl.shape)   # move biases off zero (ReLU kinks)
    X = rng.standard_normal((7, 12))
    T = rng.standard_normal((7, 5))
    Y, cache = mlp_forward(W, b, X)
    gW, gb = mlp_backward(W, b, cache, Y, T)
    h = 1e-6
    for l in range(4):
        for (i, j) in [(0, 0), (W[l].shape[0] - 1, W[l].shape[1] - 1), (1, 2)]:
            W[l][i, j] += h
            lp = mse_loss(mlp_forward(W, b, X)[0], T)
            W[l][i, j] -= 2 * h
            lm = mse_loss(mlp_forward(W, b, X)[0], T)
            W[l][i, j] += h
            fd = (lp - lm) / (2 * h)
            assert abs(fd - gW[l][i, j]) <= 1e-6 * max(1e-3, abs(fd))
        b[l][0] += h
        lp = mse_loss(mlp_forward(W, b, X)[0], T)
        b[l][0] -= 2 * h
        lm = mse_loss(mlp_forward(W, b, X)[0], T)
        b[l][0] += h
        assert abs((lp - lm) / (2 * h) - gb[l][0]) <= 1e-6 * max(1e-3, abs(gb[l][0]))


def test_oracle_mlp_forward_by_hand():
    """T-MLP: three ReLU layers and a linear output, W_l (out x in), worked by hand
    (a dropped bias, a ReLU on the output or a transposed weight changes the result)."""
    from oracle.solver import mlp_forward
    W = [np.array([[1.0, 0.0], [0.0, 1.0], [1.0, 1.0]]),
         np.eye(3),
         np.array([[1.0, 1.0, 0.0], [0.0, 0.0, 1.0], [-1.0, 0.0, 0.0]]),
         np.array([[1.0, 0.0, 2.0], [0.0, 1.0, 0.0]])]
    b = [np.array([0.0, 0.0, -1.0]), np.array([-0.5, 0.0, 0.0]), np.zeros(3), np.array([0.5, -2.5])]
    X = np.array([[1.0, 2.0], [-1.0, -1.0]])
    Y, (h, z) = mlp_forward(W, b, X)
    # row 0: h1 = (1, 2, 2), h2 = (0.5, 2, 2), h3 = (2.5, 2, 0), y = (3.0, -0.5)
    # row 1: every hidden unit is cut by the ReLU, y = b_3 (negative entry kept)
    assert Y.tolist() == [[3.0, -0.5], [0.5, -2.5]]
    assert h[1].tolist()[0] == [1.0, 2.0, 2.0] and h[3].tolist()[0] == [2.5, 2.0, 0.0]


def test_oracle_cardinal_coefficients_are_cardinal():
    """T-CARD: sum_{j in S} c_j Phi(x_k - x_j) = delta_{k, centre} for k in S."""
    from oracle.solver import knn, cardinal
    rng = np.random.default_rng(8)
    X = rng.random((400, 2))
    nb = knn(X, 32)
    c = cardinal(X, nb[:50], O.GAUSSIAN, 40.0, 0.0)   # eps*h ~ 2: well-conditioned local sets
    for i in range(50):
        P = X[nb[i]]
        A = O.phi(O.GAUSSIAN, 40.0, np.linalg.norm(P[:, None] - P[None, :], axis=2))
        e = np.zeros(32)
        e[0] = 1.0
        assert np.max(np.abs(A @ c[i] - e)) < 1e-10


def test_oracle_cardinal_regularised_by_hand():
    """T-CARD with regularisation: c = (A_S + delta I)^-1 e_1, delta = delta_rel ||A_S||_F,
    on three 1-D centres (0, 1/2, 1), Gaussian eps = 1, inverted by cofactors written out.
    A delta of delta_rel alone, a norm other than Frobenius, or a shift of the first
    diagonal entry only each miss these values."""
    from oracle.solver import cardinal
    X = np.array([[0.0], [0.5], [1.0]])
    a, b = np.exp(-0.25), np.exp(-1.0)            # Phi(1/2), Phi(1)
    fro = np.sqrt(3.0 + 4.0 * a * a + 2.0 * b * b)  # ||A_S||_F, the same for both orders
    delta_rel = 0.05
    s = 1.0 + delta_rel * fro

    def first_column_of_inverse(m):
        c11 = m[1][1] * m[2][2] - m[1][2] * m[2][1]
        c12 = -(m[1][0] * m[2][2] - m[1][2] * m[2][0])
        c13 = m[1][0] * m[2][1] - m[1][1] * m[2][0]
        det = m[0][0] * c11 + m[0][1] * c12 + m[0][2] * c13
        return np.array([c11, c12, c13]) / det

    want0 = first_column_of_inverse([[s, a, b], [a, s, a], [b, a, s]])  # S = (0, 1, 2)
    want1 = first_column_of_inverse([[s, a, a], [a, s, b], [a, b, s]])  # S = (1, 0, 2)
    c = cardinal(X, np.array([[0, 1, 2], [1, 0, 2]]), O.GAUSSIAN, 1.0, delta_rel)
    assert np.allclose(c[0], want0, rtol=1e-13, atol=0)
    assert np.allclose(c[1], want1, rtol=1e-13, atol=0)
    assert not np.allclose(c[0], first_column_of_inverse([[1 + delta_rel, a, b], [a, 1 + delta_rel, a],
                                                         [b, a, 1 + delta_rel]]), rtol=1e-6)


def test_oracle_mlp_bf16_branch_by_hand():
    """T-MLP with BF16 operands (q = bf16_round): a 2 -> 2 -> 1 network worked by hand.
    Operands round to 8 significant bits: 1.007 -> 129/128, 1.01 -> 129/128,
    0.3 -> 77/256, 2.003 -> 2, 0.7 -> 179/256, -1.3 -> -83/64; the biases and the sums
    stay FP64.  Backward: g = 2 (y - t) / y.size, each product again on rounded
    operands, ReLU mask from z."""
    from oracle.solver import bf16_round, mlp_backward, mlp_forward
    W = [np.array([[1.01, -0.5], [0.3, 2.003]]), np.array([[0.7, -1.3]])]
    b = [np.array([0.1, -0.9]), np.array([0.05])]
    X = np.array([[1.007, 0.25]])
    Y, cache = mlp_forward(W, b, X, q=bf16_round)
    x0, w11, w21 = 129 / 128, 129 / 128, 77 / 256
    z1 = np.array([x0 * w11 - 0.125 + 0.1, x0 * w21 + 0.5 - 0.9])   # second unit < 0
    assert np.allclose(cache[1][0], z1[None], rtol=1e-15, atol=1e-16)
    h1 = 127 / 128                 # bf16(0.99071...) = 1.984375 / 2
    y = h1 * (179 / 256) + 0.05
    assert abs(Y[0, 0] - y) <= 1e-15
    T = np.array([[0.5]])
    gW, gb = mlp_backward(W, b, cache, Y, T, q=bf16_round)
    g = 2.0 * (y - 0.5)                          # 0.48751..., bf16 -> 125/256
    assert abs(gb[1][0] - g) <= 1e-15
    assert np.allclose(gW[1], [[(125 / 256) * h1, 0.0]], rtol=1e-15, atol=0)
    g0 = (125 / 256) * (179 / 256)               # back through bf16 W_2; unit 2 masked
    assert np.allclose(gb[0], [g0, 0.0], rtol=1e-15, atol=0)
    gq = 175 / 512                               # bf16(g0)
    assert np.allclose(gW[0], [[gq * x0, gq * 0.25], [0.0, 0.0]], rtol=1e-15, atol=0)
    # the identity branch differs in the fourth significant digit
    Yi, _ = mlp_forward(W, b, X)
    assert abs(Yi[0, 0] - y) > 1e-4


def test_oracle_knn_by_hand():
    """Neighbour order with an exact distance tie broken by index."""
    from oracle.solver import knn
    X = np.array([[0.0, 0.0], [1.0, 0.0], [-1.0, 0.0], [0.0, 0.5], [3.0, 3.0]])
    nb = knn(X, 4)
    assert nb[0].tolist() == [0, 3, 1, 2]      # 1 and 2 tie at distance 1
    assert nb[4].tolist()[0] == 4


def test_oracle_features_by_hand():
    """T-FEAT: eps (x_j - x_i) over the neighbour list, nearest first, flattened."""
    from oracle.solver import features, knn
    X = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 2.0]])
    nb = knn(X, 3)
    assert nb.tolist() == [[0, 1, 2], [1, 0, 2], [2, 0, 1]]
    F = features(X, nb, 0.5)
    assert F.tolist() == [[0.0, 0.0, 0.5, 0.0, 0.0, 1.0],
                          [0.0, 0.0, -0.5, 0.0, -0.5, 1.0],
                          [0.0, 0.0, 0.0, -1.0, 0.5, -1.0]]


def test_oracle_adam_closed_forms():
    """T-ADAM (Kingma & Ba): with bias-corrected moments a constant gradient g moves
    every parameter by lr g / (|g| + eps) per step, whatever the step count; and
    two steps with gradients g1, g2 follow the moments written out by hand."""
    from oracle.solver import adam_step
    g = np.array([2.0, -0.5, 1e-3, 0.0])
    p = np.zeros(4)
    m = np.zeros(4)
    v = np.zeros(4)
    lr, eps = 1e-2, 1e-8
    for t in range(1, 6):
        adam_step(p, g, m, v, t, lr)
        assert np.allclose(p, -t * lr * g / (np.abs(g) + eps), rtol=1e-12, atol=0)
    g1, g2 = np.array([1.0, -3.0]), np.array([-2.0, 1.0])
    p = np.array([0.5, 0.5])
    m = np.zeros(2)
    v = np.zeros(2)
    adam_step(p, g1, m, v, 1, lr)
    adam_step(p, g2, m, v, 2, lr)
    m2 = 0.9 * 0.1 * g1 + 0.1 * g2                   # first moment after two steps
    v2 = 0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2   # second moment
    step2 = lr * (m2 / (1 - 0.9 ** 2)) / (np.sqrt(v2 / (1 - 0.999 ** 2)) + eps)
    step1 = lr * g1 / (np.abs(g1) + eps)
    assert np.allclose(p, 0.5 - step1 - step2, rtol=1e-13, atol=0)


def test_bf16_rounding_by_hand():
    """BF16 keeps 8 significant bits, ties to even: 1 + 2^-8 (a tie) -> 1; 1 + 3*2^-8 -> 1 + 2^-6;
    1 + 2^-7 is representable."""
    from oracle.solver import bf16_round
    v = bf16_round(np.array([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -7, -2.5]))
    assert v.tolist() == [1.0, 1.0 + 2 ** -6, 1.0 + 2 ** -7, -2.5]


# ------------------------------------------------------------- T-LAG -----
def _golden(name):
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    rows = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return rows


def test_lagrange_basis_reproduces_paper_error_table():
    """The Lagrange basis of the nested-grid oracle, on the paper's setting (K
    equispaced nodes on [-pi, pi], targets xi/2, |x| <= 1), reproduces the
    printed error table within 1% (K = 8, 11, 12 to every printed digit).  A
    basis with swapped indices, a missing factor or a wrong target fails."""
    from oracle import nested as ON
    for K, err in _golden("lagrange_halfwave_error.txt"):
        got = ON.lagrange_halfwave_error(int(K))
        assert abs(got / err - 1.0) < 0.01, (K, got, err)
        if int(K) in (8, 11, 12):
            assert float(f"{got:.4e}") == pytest.approx(err, rel=1e-4), (K, got, err)


def test_interp_matrix_exact_on_polynomials_and_nodes():
    """The local K-point stencil matrix reproduces every polynomial of degree < K
    at the half-node targets (closed form), is the identity selection on even
    parent nodes, and maps the symmetric grid onto itself mirrored."""
    from oracle import nested as ON
    for M, K in ((16, 8), (32, 8), (24, 12), (20, 4)):
        P = ON.interp_matrix(M, K)
        j = np.arange(-M // 2, M // 2 + 1, dtype=np.float64)
        for deg in range(K):
            assert np.allclose(P @ (j ** deg), (j / 2.0) ** deg, rtol=1e-12, atol=1e-9 * (M ** deg))
        for kp in range(0, M + 1):
            k = kp - M // 2
            if k % 2 == 0:
                row = np.zeros(M + 1)
                row[k // 2 + M // 2] = 1.0
                assert np.array_equal(P[kp], row)
        assert np.allclose(P[::-1, ::-1], P, rtol=0, atol=1e-15)


def test_nested_depth2_equals_shared_grid():
    """With D = 2 only level 2 couples, and its grid and coefficients are those of
    the shared grid: the nested product equals the shared-grid product."""
    from oracle import nested as ON
    rng = np.random.default_rng(3)
    X = rng.random((600, 2))
    lam = rng.standard_normal(600)
    T = O.tree(X, np.zeros(2), 1.0, 2)
    wcs = ON.coeffs_levels(O.IMQ, 2.0, 2, 16, 4.0, 4.5, 1.0, 2)
    wc = O.coeffs_sampled(O.IMQ, 2.0, 2, 16, 4.0, 4.5, 1.0)
    assert np.array_equal(wcs[2], wc)
    assert rel(ON.fmm(T, lam, O.IMQ, 2.0, wcs, 16, 4.0, 8), O.fmm(T, lam, O.IMQ, 2.0, wc, 16, 4.0)) < 1e-14


@pytest.mark.parametrize("d,N,D,kernel,eps,M,K", [
    (1, 120, 4, O.IMQ, 2.0, 16, 8),
    (2, 150, 3, O.IMQ, 2.0, 16, 8),
    (2, 120, 4, O.GAUSSIAN, 3.0, 16, 6),
    (3, 90, 3, O.IMQ, 2.0, 8, 4),
])
def test_nested_fmm_equals_pairwise_chains(d, N, D, kernel, eps, M, K):
    """The nested FMM (box expansions, M2M by interpolation, IL_l coupling, L2L by
    anterpolation) equals the pair-by-pair sum built from one-dimensional phase
    chains, with pairs classified from their box coordinates."""
    from oracle import nested as ON
    rng = np.random.default_rng(7 * N + d)
    X = rng.random((N, d))
    lam = rng.standard_normal(N)
    T = O.tree(X, np.zeros(d), 1.0, D)
    wcs = ON.coeffs_levels(kernel, eps, d, M, 4.0, 4.5, 1.0, D)
    u = ON.fmm(T, lam, kernel, eps, wcs, M, 4.0, K)
    up = ON.fmm_pairwise(X, lam, np.zeros(d), 1.0, D, kernel, eps, wcs, M, 4.0, K)
    assert rel(u, up) < 1e-13


def test_nested_fmm_converges_to_level_kernels():
    """As K grows the interpolated phases become exact, and the nested product
    tends to near Phi + far K_l (each far pair with the band-limited kernel of
    the level that couples it); against the direct sum the error is bounded by
    max |K_l - Phi| * sum |lambda| plus the interpolation error."""
    from oracle import nested as ON
    d, N, D, M, eps = 2, 900, 4, 24, 2.0
    rng = np.random.default_rng(21)
    X = rng.random((N, d))
    lam = rng.standard_normal(N)
    T = O.tree(X, np.zeros(d), 1.0, D)
    wcs = ON.coeffs_levels(O.IMQ, eps, d, M, 4.0, 4.5, 1.0, D)
    ud = O.direct(X, lam, O.IMQ, eps)
    kerr = ON.kernel_levels_error(O.IMQ, eps, d, M, 4.0, wcs, 1.0, D)
    errs = []
    for K in (4, 8, 12):
        u = ON.fmm(T, lam, O.IMQ, eps, wcs, M, 4.0, K)
        errs.append(np.max(np.abs(u - ud)))
    assert errs[0] > errs[1] >= errs[2] * 0.5
    assert errs[2] <= 1.05 * kerr * np.sum(np.abs(lam))


# ------------------------------------------------------ new points -------
def test_evaluate_at_centres_equals_product():
    """Evaluating at copies of some centres reproduces the product at those
    centres: the copies fall in the same boxes, carry zero coefficients and
    change neither the lists nor any expansion."""
    rng = np.random.default_rng(12)
    X = rng.random((500, 2))
    lam = rng.standard_normal(500)
    wc = O.coeffs_sampled(O.IMQ, 2.0, 2, 16, 4.0, 4.5, 1.0)
    T = O.tree(X, np.zeros(2), 1.0, 3)
    u = O.fmm(T, lam, O.IMQ, 2.0, wc, 16, 4.0)
    pick = rng.choice(500, 40, replace=False)
    s = O.fmm_evaluate(X, lam, X[pick], np.zeros(2), 1.0, 3, O.IMQ, 2.0, wc, 16, 4.0)
    assert np.max(np.abs(s - u[pick])) <= 1e-14 * np.max(np.abs(u))


@pytest.mark.parametrize("kernel,eps,alpha", [(O.IMQ, 2.0, 4.5), (O.GAUSSIAN, 3.0, 0.0),
                                              (O.MQ, 1.0, 4.5)])
def test_evaluate_within_lemma_bound(kernel, eps, alpha):
    """At new points the evaluation differs from the direct interpolant
    sum_j lambda_j Phi(y - x_j) by at most max_far |K - Phi| * sum |lambda|
    (scaled Lemma, Eq. (33))."""
    rng = np.random.default_rng(13)
    X = rng.random((800, 2))
    Y = rng.random((300, 2))
    lam = rng.standard_normal(800)
    M, L = 24, (3.0 if kernel == O.GAUSSIAN else 4.0)
    wc = O.coeffs_sampled(kernel, eps, 2, M, L, alpha, 1.0)
    s = O.fmm_evaluate(X, lam, Y, np.zeros(2), 1.0, 3, kernel, eps, wc, M, L)
    Z = np.concatenate([X, Y])
    sd = O.direct(Z, np.concatenate([lam, np.zeros(300)]), kernel, eps, np.arange(800, 1100))
    r = rng.uniform(-1, 1, (6000, 2))
    r = r[np.max(np.abs(r), axis=1) >= 1.0 / 8]
    kerr = np.max(np.abs(O.kernel_K(wc, 2, M, L, r) - O.phi(kernel, eps, np.linalg.norm(r, axis=1))))
    assert np.max(np.abs(s - sd)) <= kerr * np.sum(np.abs(lam))
    assert np.max(np.abs(s - sd)) > 0.0
