"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test names the passage it checks.  None of them re-derives an expected
value from the oracle's own formulas: they use closed forms, brute-force
exact diagonalisation, identities of the Kronecker/partial-trace calculus,
finite differences, and the paper's inequalities.
"""
import itertools

import numpy as np
import pytest

import lrh_gen as g
from oracle import dual, exact
from oracle.poset import Poset

L = g.lattices


def rand_herm_msgs(P, I, rng, scale):
    nu = np.zeros((I, P.msg_total), np.complex128)
    for p in range(P.n_pairs):
        Df = int(P.D[P.pair_child[p]])
        for i in range(I):
            A = L.random_hermitian(rng, Df, scale)
            nu[i, P.msg_off[p]:P.msg_off[p] + Df * Df] = A.reshape(-1)
    return nu


def converge(P, h, betas=None, iters=300, I=1):
    betas = betas or [2.0 ** s for s in range(0, 15)]
    st = dual.run_nesterov(P, h, betas, iters, n_instances=I)
    return dual.dual_value(P, h, st.nu), st


# ---------------------------------------------------------------- exact solvers
@pytest.mark.parametrize("n,seed", [(3, 1), (5, 2), (8, 3), (11, 4)])
def test_free_fermion_matches_exact_diagonalisation(n, seed):
    p = L.tfim_chain(n, seed)
    assert abs(exact.ground_energy(p) - exact.tfim_free_fermion_e0(p.meta["J"], p.meta["h"])) < 1e-9


# ---------------------------------------------------------------- Kronecker conventions
def test_embed_matches_explicit_kron():
    rng = np.random.default_rng(0)
    A = L.random_hermitian(rng, 2)
    B = L.random_hermitian(rng, 4)
    I2 = np.eye(2)
    # 3-site region (s0,s1,s2), first site most significant
    assert np.allclose(dual.embed(A, [0], 3), np.kron(A, np.kron(I2, I2)))
    assert np.allclose(dual.embed(A, [2], 3), np.kron(np.kron(I2, I2), A))
    assert np.allclose(dual.embed(B, [0, 1], 3), np.kron(B, I2))
    assert np.allclose(dual.embed(B, [1, 2], 3), np.kron(I2, B))
    # non-adjacent positions: B acting on (s0, s2); check on product operators
    P, Q = L.random_hermitian(rng, 2), L.random_hermitian(rng, 2)
    assert np.allclose(dual.embed(np.kron(P, Q), [0, 2], 3), np.kron(np.kron(P, I2), Q))


def test_partial_trace_is_adjoint_of_embedding():
    rng = np.random.default_rng(1)
    for k, pos in [(2, (0,)), (2, (1,)), (3, (0, 2)), (4, (1, 3)), (4, (0, 1, 2))]:
        D, Df = 2 ** k, 2 ** len(pos)
        rho = L.random_hermitian(rng, D)
        nu = L.random_hermitian(rng, Df)
        lhs = np.trace(rho @ dual.embed(nu, pos, k))
        rhs = np.trace(dual.partial_trace(rho, pos, k) @ nu)
        assert abs(lhs - rhs) < 1e-12
    # product state: Tr_2 (A (x) B) = A Tr B
    A, B = L.random_hermitian(rng, 2), L.random_hermitian(rng, 2)
    assert np.allclose(dual.partial_trace(np.kron(A, B), (0,), 2), A * np.trace(B))
    assert np.allclose(dual.partial_trace(np.kron(A, B), (1,), 2), B * np.trace(A))


# ---------------------------------------------------------------- poset (Fig. 1, Sec. 4.2)
def test_interval_poset_matches_fig1_chain_of_three():
    P = Poset(L.interval_regions(3, 3))
    reg = {r: i for i, r in enumerate(P.regions)}
    kids = {P.regions[e]: sorted(P.regions[f] for f in P.children[e]) for e in range(len(P.regions))}
    assert kids[(0, 1, 2)] == [(0, 1), (1, 2)]
    assert kids[(0, 1)] == [(0,), (1,)]
    assert kids[(1, 2)] == [(1,), (2,)]
    assert kids[(1,)] == []
    # the implied constraint (0,1,2) -> (1,) is not a covering pair
    assert (reg[(0, 1, 2)], reg[(1,)]) not in set(zip(P.pair_parent.tolist(), P.pair_child.tolist()))


def test_plaquette_poset_children():
    P = Poset(L.xxz_triangular(3, 1).regions)
    for e, r in enumerate(P.regions):
        if len(r) == 4:
            assert len(P.children[e]) == 5          # 4 sides + the (1,1) diagonal
        if len(r) == 2:
            assert len(P.children[e]) == 2
    P = Poset(L.j1j2_square(3, J2s=(0.5,)).regions)
    assert all(len(P.children[e]) == 4 for e, r in enumerate(P.regions) if len(r) == 4)


def test_lambda_and_gamma_hand_values():
    # level 1, open chain: max degree 2 -> Lambda = Delta + d = 4 (Lipschitz lemma)
    assert Poset(L.tfim_chain(16).regions).lipschitz_lambda() == 4.0
    # periodic square lattice: degree 4 -> 6
    assert Poset(L.heisenberg_square(4).regions).lipschitz_lambda() == 6.0
    # intervals L >= 4 on a long chain: interior non-top e has m_e = 2 + 2,
    # its child f has m_f = 4, D_e / D_f = 2  ->  4 + 4 * 2 = 12   (Thm 7)
    assert Poset(L.interval_regions(20, 4)).lipschitz_lambda() == 12.0
    # Gamma = sum log D: 15 edges (log 4) + 16 nodes (log 2) = 46 log 2
    assert abs(Poset(L.tfim_chain(16).regions).gamma() - 46 * np.log(2)) < 1e-12


# ---------------------------------------------------------------- dual value
def test_anderson_value_at_zero_messages_tfim():
    # theta = h at nu = 0; lambda_min(-J ZZ) = -J, lambda_min(-h X) = -h (Sec. 3.1 Anderson bound)
    p = L.tfim_chain(16, 1001)
    P = Poset(p.regions)
    q0 = dual.dual_value(P, dual.local_terms(p, P), dual.zeros_messages(P, 1))[0]
    assert abs(q0 - (-sum(p.meta["J"]) - sum(p.meta["h"]))) < 1e-12


@pytest.mark.parametrize("builder", [
    lambda: L.random_chain(6, 11, L=2),
    lambda: L.random_chain(7, 12, L=3),
    lambda: L.random_graph_problem(6, [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4), (4, 5), (5, 0)], 13),
    lambda: L.j1j2_square(3, J2s=(0.3,)),
    lambda: L.xxz_triangular(3, 2),
])
def test_weak_duality_random_messages(builder):
    """Q(nu) <= E_0 for every Hermitian nu (Sec. 4.1, weak duality)."""
    p = builder()
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    rng = np.random.default_rng(5)
    E0 = np.array([exact.ground_energy(p, i) for i in range(p.n_instances)])
    worst = -np.inf
    for scale in [0.3, 1.0, 3.0]:
        for _ in range(4):
            nu = rand_herm_msgs(P, p.n_instances, rng, scale)
            q = dual.dual_value(P, h, nu)
            worst = max(worst, float(np.max(q - E0)))
    assert worst <= 1e-10


# ---------------------------------------------------------------- gradients
@pytest.mark.parametrize("builder,beta", [
    (lambda: L.random_chain(5, 21, L=2), 2.0),
    (lambda: L.random_chain(6, 22, L=3), 5.0),
    (lambda: L.j1j2_square(3, J2s=(0.5,)), 1.5),
])
def test_smoothed_gradient_matches_finite_differences(builder, beta):
    """grad_{nu_{e->f}} Q_beta = rho_f - Tr_{e\\f} rho_e (Sec. 4.1.2, Sec. 4.2)."""
    p = builder()
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    rng = np.random.default_rng(3)
    nu = rand_herm_msgs(P, 1, rng, 0.5)
    res = dual.region_pass(P, h, nu, "smooth", beta=beta)
    for _ in range(3):
        d = rand_herm_msgs(P, 1, rng, 1.0)
        eps = 1e-5
        fd = (dual.smoothed_value(P, h, nu + eps * d, beta) - dual.smoothed_value(P, h, nu - eps * d, beta)) / (2 * eps)
        an = np.real(np.vdot(d[0], res.grad[0]))
        assert abs(fd[0] - an) <= 1e-7 * max(1.0, abs(an))


def test_subgradient_matches_finite_differences_when_nondegenerate():
    """At a point with non-degenerate ground states Q is differentiable and the
    subgradient mu_f - Tr mu_e is its gradient (Sec. 4.1.1)."""
    p = L.random_chain(5, 31, L=2)
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    rng = np.random.default_rng(4)
    nu = rand_herm_msgs(P, 1, rng, 0.5)
    res = dual.region_pass(P, h, nu, "ground")
    d = rand_herm_msgs(P, 1, rng, 1.0)
    eps = 1e-6
    fd = (dual.dual_value(P, h, nu + eps * d) - dual.dual_value(P, h, nu - eps * d)) / (2 * eps)
    assert abs(fd[0] - np.real(np.vdot(d[0], res.grad[0]))) < 1e-6


# ---------------------------------------------------------------- smoothing lemma
def test_smoothing_sandwich():
    """F_beta <= lambda_min <= F_beta + log D / beta per region, hence
    Q_beta <= Q <= Q_beta + Gamma / beta (smoothing-error lemmas, Sec. 4.1.2, 4.2)."""
    p = L.random_chain(6, 41, L=3)
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    rng = np.random.default_rng(6)
    nu = rand_herm_msgs(P, 1, rng, 1.0)
    for beta in [0.5, 4.0, 64.0]:
        res = dual.region_pass(P, h, nu, "smooth", beta=beta)
        F, lm = res.value[0], res.lam_min[0]
        assert np.all(F <= lm + 1e-12)
        assert np.all(lm <= F + np.log(P.D) / beta + 1e-12)
        q, qb = dual.dual_value(P, h, nu)[0], dual.smoothed_value(P, h, nu, beta)[0]
        assert qb <= q + 1e-12 and q <= qb + P.gamma() / beta + 1e-12


# ---------------------------------------------------------------- invariants
def test_messages_stay_hermitian_and_traceless():
    """Zero-initialised messages stay traceless: every gradient component is a
    difference of two unit-trace states (appendix, proof of the Lipschitz lemma)."""
    p = L.random_chain(6, 51, L=3)
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    st = dual.run_nesterov(P, h, [1.0, 4.0], 20)
    sg = dual.run_subgradient(P, h, 20)
    for nu in (st.nu, st.zeta, sg.nu):
        for q in range(P.n_pairs):
            Df = int(P.D[P.pair_child[q]])
            M = nu[0, P.msg_off[q]:P.msg_off[q] + Df * Df].reshape(Df, Df)
            assert abs(np.trace(M)) < 1e-12
            assert np.allclose(M, M.conj().T, atol=1e-13)


def test_subgradient_component_norm_bound():
    """||g_{e->f}||_F^2 <= 2 (difference of two density matrices; proof of Thm 4)."""
    p = L.random_chain(6, 61, L=3)
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    rng = np.random.default_rng(7)
    for scale in [0.1, 1.0, 5.0]:
        res = dual.region_pass(P, h, rand_herm_msgs(P, 1, rng, scale), "ground")
        for q in range(P.n_pairs):
            Df = int(P.D[P.pair_child[q]])
            gq = res.grad[0, P.msg_off[q]:P.msg_off[q] + Df * Df]
            assert np.sum(np.abs(gq) ** 2) <= 2 + 1e-12


def test_nesterov_theta_sequence():
    """theta_{k+1} solves (1 - theta_{k+1}) / theta_{k+1}^2 = 1 / theta_k^2
    (the recurrence of Alg. 2) and theta_k <= 2 / (k + 2)."""
    th = 1.0
    for k in range(200):
        nt = dual.next_theta(th)
        assert abs((1 - nt) / nt ** 2 - 1 / th ** 2) < 1e-9 / th ** 2
        assert th <= 2.0 / (k + 2) + 1e-15
        th = nt


# ---------------------------------------------------------------- exact relaxations
def test_level1_exact_for_separable_hamiltonian_on_edges():
    """H = sum_i C_i written as edge terms A_i (x) 1 + 1 (x) B_{i+1}: every
    locally consistent mu gives sum <mu_i, C_i> >= sum lambda_min(C_i) = E_0, so
    f_1 = E_0 although Q(0) < E_0."""
    rng = np.random.default_rng(71)
    n = 6
    A = [L.random_hermitian(rng, 2) for _ in range(n)]
    B = [L.random_hermitian(rng, 2) for _ in range(n)]
    ts, tm = [], []
    for i in range(n - 1):
        ts.append((i, i + 1)); tm.append((np.kron(A[i], np.eye(2)) + np.kron(np.eye(2), B[i + 1]))[None])
    p = g.Problem(n, L.level1_regions(n, [(i, i + 1) for i in range(n - 1)]), ts, tm)
    E0 = exact.ground_energy(p)
    C = [(A[i] if i < n - 1 else 0) + (B[i] if i > 0 else 0) for i in range(n)]
    assert abs(E0 - sum(np.linalg.eigvalsh(c)[0] for c in C)) < 1e-10
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    assert dual.dual_value(P, h, dual.zeros_messages(P, 1))[0] < E0 - 0.1
    q, _ = converge(P, h)
    assert q[0] <= E0 + 1e-9 and (E0 - q[0]) / n < 1e-4


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_level1_exact_for_commuting_tree(seed):
    """Thm 2: level 1 is exact for commuting 2-local Hamiltonians on trees."""
    p = L.commuting_tree(7, seed)
    H = [exact._embed_full(m[0], s, p.n_sites).toarray() for s, m in zip(p.term_sites, p.term_mats)]
    for a, b in itertools.combinations(H, 2):
        assert np.abs(a @ b - b @ a).max() < 1e-10     # generator really commutes
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    E0 = exact.ground_energy(p)
    q, _ = converge(P, h)
    assert q[0] <= E0 + 1e-9 and (E0 - q[0]) / p.n_sites < 2e-4


@pytest.mark.parametrize("seed", [5, 6])
def test_level1_exact_for_classical_tree(seed):
    """Diagonal Hamiltonian on a tree: M_c(T) = L_c(T) (Sec. 3.1)."""
    p = L.classical_tree(8, seed)
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    E0 = exact.ground_energy(p)
    q, _ = converge(P, h)
    assert q[0] <= E0 + 1e-9 and (E0 - q[0]) / p.n_sites < 2e-4


def test_exact_for_frustration_free():
    """Frustration-free H: E_0 = sum lambda_min(h_e) = Anderson bound (Sec. 3.1)."""
    p = L.frustration_free_chain(6, 81, L=2)
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    E0 = exact.ground_energy(p)
    assert abs(dual.dual_value(P, h, dual.zeros_messages(P, 1))[0] - E0) < 1e-9
    q, _ = converge(P, h, iters=50)
    assert abs(q[0] - E0) < 1e-6


def test_whole_system_cluster_is_exact():
    """A cluster family containing the whole chain gives E_0 (Sec. 3.2)."""
    p = L.random_chain(5, 91, L=5)
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    E0 = exact.ground_energy(p)
    q, _ = converge(P, h, betas=[2.0 ** s for s in range(0, 16)], iters=300)
    assert q[0] <= E0 + 1e-9 and (E0 - q[0]) / p.n_sites < 2e-4


def test_not_exact_for_generic_frustrated_tree():
    """Contrast case: a generic non-commuting chain keeps a visible gap at
    level 1, so the exactness tests above discriminate."""
    p = L.random_chain(6, 101, L=2, scale=1.0)
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    E0 = exact.ground_energy(p)
    q, _ = converge(P, h)
    assert (E0 - q[0]) / p.n_sites > 1e-3


def test_interval_hierarchy_monotone_and_one_over_t():
    """Growing the intervals tightens the bound (Sec. 3.2): f_2 <= f_3 <= f_4 <= E_0;
    and with 2||h|| <= 1, (E_0 - f_t)/n <= 1/t (Sec. 3.3)."""
    n = 8
    rng = np.random.default_rng(111)
    ts, tm = [], []
    for i in range(n - 1):
        A = L.random_hermitian(rng, 4)
        A = A / (2 * np.abs(np.linalg.eigvalsh(A)).max())      # 2 ||h|| = 1
        ts.append((i, i + 1)); tm.append(A[None])
    E0 = exact.ground_energy(g.Problem(n, L.interval_regions(n, 2), ts, tm))
    vals = []
    for t in (2, 3, 4):
        p = g.Problem(n, L.interval_regions(n, t), ts, tm)
        P = Poset(p.regions)
        q, _ = converge(P, dual.local_terms(p, P), iters=200)
        vals.append(q[0])
        assert (E0 - q[0]) / n <= 1.0 / t
    tol = 5e-4 * n
    assert vals[0] <= vals[1] + tol and vals[1] <= vals[2] + tol and vals[2] <= E0 + 1e-9
    assert vals[2] - vals[0] > 10 * tol      # the tightening is visible


def test_subgradient_bound_below_e0_tfim():
    """Alg. 1 on the TFIM chain (n = 16): q_best <= f_1 <= E_0 (free-fermion E_0)
    and it improves on the Anderson value."""
    p = L.tfim_chain(16, 1001)
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    E0 = exact.tfim_free_fermion_e0(p.meta["J"], p.meta["h"])
    st = dual.run_subgradient(P, h, 300)
    q0 = dual.dual_value(P, h, dual.zeros_messages(P, 1))[0]
    assert st.q_best[0] <= E0 and st.q_best[0] > q0 + 1.0


# ---------------------------------------------------------------- Alg. 2 update form, by hand
def _classical_edge_problem():
    """One edge (0, 1) with a diagonal term and diagonal site terms: every theta, Gibbs state
    and gradient stays diagonal, and with traceless diagonal messages x Z (edge -> site 0) and
    y Z (edge -> site 1) the whole iteration reduces to two real numbers."""
    e = np.array([0.3, -1.1, 0.7, 0.2])        # basis |00>, |01>, |10>, |11>
    h0 = np.array([0.25, -0.4])
    h1 = np.array([-0.1, 0.35])
    p = g.Problem(2, [(0, 1), (0,), (1,)], [(0, 1), (0,), (1,)],
                  [np.diag(e).astype(complex)[None], np.diag(h0).astype(complex)[None],
                   np.diag(h1).astype(complex)[None]])
    return p, e, h0, h1


def _hand_gibbs(diag, beta):
    w = [np.exp(-beta * (v - min(diag))) for v in diag]
    z = sum(w)
    return [x / z for x in w], min(diag) - np.log(z) / beta


def _hand_smoothed_pass(x, y, e, h0, h1, beta):
    """Q_beta and the Z-components of g_{e->0}, g_{e->1} at messages x Z, y Z, from scalars
    only: theta_e[ab] = e_ab - x z_a - y z_b (z_0 = 1, z_1 = -1), theta_0 = h0 + x Z,
    theta_1 = h1 + y Z; Gibbs states of diagonal matrices are softmaxes of the diagonal."""
    z = (1.0, -1.0)
    te = [e[2 * a + b] - x * z[a] - y * z[b] for a in (0, 1) for b in (0, 1)]
    re, fe = _hand_gibbs(te, beta)
    r0, f0 = _hand_gibbs([h0[0] + x, h0[1] - x], beta)
    r1, f1 = _hand_gibbs([h1[0] + y, h1[1] - y], beta)
    marg0 = re[0] + re[1]            # <0| Tr_1 rho_e |0>
    marg1 = re[0] + re[2]            # <0| Tr_0 rho_e |0>
    return fe + f0 + f1, r0[0] - marg0, r1[0] - marg1


def test_nesterov_three_steps_by_hand():
    """Alg. 2 from nu = zeta = 0, theta_0 = 1: eta = (1 - theta) nu + theta zeta, gradient at
    eta, zeta += g / (theta L_hat), nu = (1 - theta) nu + theta zeta, theta update.  The first
    two iterations have eta = nu = zeta; the third is the first where eta differs from nu, so
    three steps fix the whole update."""
    p, e, h0, h1 = _classical_edge_problem()
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    beta, lhat = 3.0, 2.5
    st = dual.NesterovState(nu=dual.zeros_messages(P, 1), zeta=dual.zeros_messages(P, 1))
    nx = ny = zx = zy = 0.0
    th = 1.0
    for _ in range(3):
        ex, ey = (1 - th) * nx + th * zx, (1 - th) * ny + th * zy
        q, gx, gy = _hand_smoothed_pass(ex, ey, e, h0, h1, beta)
        zx, zy = zx + gx / (th * lhat), zy + gy / (th * lhat)
        nx, ny = (1 - th) * nx + th * zx, (1 - th) * ny + th * zy
        th = (np.sqrt(th ** 4 + 4 * th ** 2) - th ** 2) / 2
        res = dual.nesterov_step(P, h, st, beta, lhat)
        assert abs(res.value.sum() - q) < 1e-12
        for arr, (a, b) in ((st.nu, (nx, ny)), (st.zeta, (zx, zy))):
            want = np.array([a, 0, 0, -a, b, 0, 0, -b], complex)     # x Z then y Z, row-major
            assert np.abs(arr[0] - want).max() < 1e-12
        assert abs(st.theta - th) < 1e-15
    assert abs(nx - zx) > 1e-3          # the three steps did separate nu from zeta


def test_nesterov_rate_of_the_accelerated_corollary():
    """Thm 5 (its proof cites Tseng's corollary): Q_beta* - Q_beta(nu_T) <= 2 L_hat R^2 / (T+1)^2
    with L_hat = beta Lambda / 2 and R = ||nu_beta* - nu_0||.  On this chain plain gradient ascent
    with step 1/L_hat exceeds the bound by up to 2x at T = 40 .. 160, so the test fixes the
    accelerated form, not only convergence."""
    p = L.random_chain(5, 5, L=2, scale=1.0)
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    beta = 8.0
    lhat = beta * P.lipschitz_lambda() / 2
    st = dual.NesterovState(nu=dual.zeros_messages(P, 1), zeta=dual.zeros_messages(P, 1))
    q = []
    for _ in range(4000):
        dual.nesterov_step(P, h, st, beta, lhat)
        if len(q) < 160:
            q.append(dual.smoothed_value(P, h, st.nu, beta)[0])
    qstar = dual.smoothed_value(P, h, st.nu, beta)[0]
    R2 = float(np.sum(np.abs(st.nu) ** 2))
    for T in (5, 10, 20, 40, 80, 160):
        assert qstar - q[T - 1] <= 2 * lhat * R2 / (T + 1) ** 2


# ---------------------------------------------------------------- Alg. 1 step rule, by hand
def test_subgradient_inv_sqrt_steps_by_hand():
    """Alg. 1 with alpha_t = alpha / sqrt(t + 1) on the classical edge: ground states of
    diagonal matrices are basis states, the degenerate site Hamiltonian at x = 0 gives the
    uniform mixture I/2, and every update is nu += alpha_t (mu_f - Tr mu_e).  Six steps
    computed from scalars fix the rule (1/(t+1) or a constant step differ from t = 2 on),
    q_best and nu_best; a field on site 1 against the edge's ground state keeps the
    subgradient from vanishing after the first step."""
    p, e, _, _ = _classical_edge_problem()
    f1 = np.array([-0.45, 0.6])     # site-1 field against the edge's ground state |01>: frustration
    p = g.Problem(2, [(0, 1), (0,), (1,)], [(0, 1), (1,)],
                  [np.diag(e).astype(complex)[None], np.diag(f1).astype(complex)[None]])
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    alpha, tol = 0.7, 1e-9
    st = dual.SubgradientState(nu=dual.zeros_messages(P, 1))
    x = y = 0.0
    qb, xb, yb = -np.inf, 0.0, 0.0
    z = (1.0, -1.0)

    def site_ground(d0, d1):       # <0|mu|0> for diag(d0, d1): 1, 0, or 1/2 when degenerate
        if abs(d1 - d0) <= tol * max(1.0, np.hypot(d0, d1)):
            return 0.5
        return 1.0 if d0 < d1 else 0.0

    for t in range(6):
        te = [e[2 * a + b] - x * z[a] - y * z[b] for a in (0, 1) for b in (0, 1)]
        k = int(np.argmin(te))
        q = min(te) - abs(x) + min(f1[0] + y, f1[1] - y)
        gx = site_ground(x, -x) - (1.0 if k in (0, 1) else 0.0)
        gy = site_ground(f1[0] + y, f1[1] - y) - (1.0 if k in (0, 2) else 0.0)
        if q > qb:
            qb, xb, yb = q, x, y
        at = alpha / np.sqrt(t + 1.0)
        x, y = x + at * gx, y + at * gy
        dual.subgradient_step(P, h, st, "sqrt", alpha, tol)
        assert abs(st.history[-1][0] - q) < 1e-12
        assert np.abs(st.nu[0] - np.array([x, 0, 0, -x, y, 0, 0, -y])).max() < 1e-12
        assert abs(st.q_best[0] - qb) < 1e-12
        assert np.abs(st.nu_best[0] - np.array([xb, 0, 0, -xb, yb, 0, 0, -yb])).max() < 1e-12


# ---------------------------------------------------------------- degenerate ground spaces
@pytest.mark.parametrize("spectrum,mult", [((-1, -1, 1, 1), 2), ((-2, -2, -2, 0.5), 3), ((-1, 0, 0.5, 2), 1)])
def test_ground_mixture_is_the_normalised_ground_projector(spectrum, mult):
    """Alg. 1's sampled ground state, read as the uniform mixture over the ground space, is the
    ground-space projector divided by its rank, whatever eigenbasis the solver returns inside
    the degenerate space: theta = U diag(spectrum) U^dagger has mixture U P U^dagger / mult."""
    rng = np.random.default_rng(17)
    U = L.random_unitary(rng, 4)
    th = U @ np.diag(np.array(spectrum, float)) @ U.conj().T
    p = g.Problem(2, [(0, 1)], [(0, 1)], [(0.5 * (th + th.conj().T))[None]])
    P = Poset(p.regions)
    res = dual.region_pass(P, dual.local_terms(p, P), dual.zeros_messages(P, 1), "ground", tol=1e-9)
    proj = np.diag([1.0 if s == min(spectrum) else 0.0 for s in spectrum])
    assert np.abs(res.states[2][0, 0] - U @ proj @ U.conj().T / mult).max() < 1e-12
    assert abs(res.value[0, 0] - min(spectrum)) < 1e-12


def test_near_degenerate_level_outside_the_tolerance_is_excluded():
    """A level 1e-6 above lambda_min is outside tol = 1e-9 * max(1, ||theta||_F): pure state."""
    th = np.diag([-1.0, -1.0 + 1e-6, 0.3, 0.9]).astype(complex)
    p = g.Problem(2, [(0, 1)], [(0, 1)], [th[None]])
    P = Poset(p.regions)
    res = dual.region_pass(P, dual.local_terms(p, P), dual.zeros_messages(P, 1), "ground", tol=1e-9)
    assert np.abs(res.states[2][0, 0] - np.diag([1.0, 0, 0, 0])).max() < 1e-12


# ---------------------------------------------------------------- sampled pass = full pass
@pytest.mark.parametrize("builder,mode", [(lambda: L.xxz_triangular(4, 3), "smooth"),
                                          (lambda: L.random_chain(7, 3, L=4), "smooth"),
                                          (lambda: L.random_chain(6, 4, L=3), "ground")])
def test_sampled_pass_equals_full_pass(builder, mode):
    """The per-sample evaluation used at benchmark sizes is the full region pass restricted to
    the sampled pairs (same values, gradients and theta norms)."""
    p = builder()
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    rng = np.random.default_rng(9)
    nu = rand_herm_msgs(P, p.n_instances, rng, 0.8)
    full = dual.region_pass(P, h, nu, mode, beta=3.0, tol=1e-9)
    th = dual.assemble(P, h, nu)
    qs = rng.integers(0, P.n_pairs, 12)
    ins = rng.integers(0, p.n_instances, 12)
    grads, vals, norms = dual.sampled_pass(p, P, nu, qs, ins, mode, beta=3.0, tol=1e-9)
    for q, i, gq in zip(qs, ins, grads):
        Df = int(P.D[P.pair_child[q]])
        assert np.abs(full.grad[i, P.msg_off[q]:P.msg_off[q] + Df * Df].reshape(Df, Df) - gq).max() < 1e-12
    for (i, e), v in vals.items():
        assert abs(full.value[i, e] - v) < 1e-12
        kk = int(P.k[e])
        assert abs(np.linalg.norm(th[kk][i, P.local_index[e]]) - norms[(i, e)]) < 1e-12
