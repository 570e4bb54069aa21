"""Pins of the FP64 oracle against things other than itself.

Each test checks the oracle against what the paper or plain mathematics fixes:
the paper's worked unfolding example, dense brute-force reconstruction with
numpy n-mode products, the CP identity of a Kruskal core, central finite
differences of the sampled loss, the textbook matrix-factorisation special
case, descent for small steps, permutation invariants of the sampler and the
library stable sort.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed):
    return np.random.default_rng(seed)


def _random_model(shape, ranks, R, seed, scale=1.0):
    g = _rng(seed)
    A = [scale * g.standard_normal((I, J)) for I, J in zip(shape, ranks)]
    B = [scale * g.standard_normal((J, R)) for J in ranks]
    return O.Model(shape, ranks, R, A, B)


def _random_batch(shape, m, seed, distinct=True):
    g = _rng(seed)
    if distinct:
        cells = int(np.prod(shape))
        lin = g.choice(cells, size=m, replace=False)
        coords = np.stack(np.unravel_index(lin, shape, order="F"), axis=1).astype(np.int32)
    else:
        coords = np.stack([g.integers(0, I, size=m) for I in shape], axis=1).astype(np.int32)
    x = g.standard_normal(m).astype(np.float32)
    return coords, x


def _dense_reconstruction(G, A):
    """G x_1 A1 x_2 A2 ... x_N AN by successive n-mode products (Def. 4, Def. 6),
    standard reading (Kolda & Bader): contract core index j_n with A_n[i_n, j_n]."""
    X = G
    for n, a in enumerate(A):
        X = np.tensordot(a, X, axes=([1], [n]))      # new axis 0 = i_n
        X = np.moveaxis(X, 0, n)
    return X


def _kruskal_core_numpy(B):
    """Core sum_r b1_r o ... o bN_r written with numpy outer products."""
    R = B[0].shape[1]
    G = None
    for r in range(R):
        t = B[0][:, r]
        for b in B[1:]:
            t = np.multiply.outer(t, b[:, r])
        G = t if G is None else G + t
    return G


# ---------------------------------------------------------------------------
# Index conventions
# ---------------------------------------------------------------------------

def test_unfolding_matches_paper_worked_example():
    rows = []
    dims = None
    with open(os.path.join(GOLDEN, "unfolding_worked_example.txt")) as fh:
        for line in fh:
            if line.startswith("# dims:"):
                parts = line.split()
                dims = [int(parts[2]), int(parts[3]), int(parts[4])]
                mode = int(parts[6])
            elif line.strip() and not line.startswith("#"):
                rows.append([int(v) for v in line.split()])
    assert dims == [3, 3, 3] and len(rows) == 4
    for i1, i2, i3, col in rows:
        c = O.unfold_column(dims, mode - 1, [i1 - 1, i2 - 1, i3 - 1])
        assert c + 1 == col
        # the digit decoder used inside the oracle is the inverse of that map
        d = O.unfold_digits(dims, mode - 1, c)
        assert list(d[1:]) == [i2 - 1, i3 - 1]


@pytest.mark.parametrize("ranks,n", [((3, 4, 5), 0), ((3, 4, 5), 1), ((3, 4, 5), 2), ((2, 3, 2, 4), 2)])
def test_unfold_digits_roundtrip(ranks, n):
    P = int(np.prod(ranks)) // ranks[n]
    seen = set()
    for c in range(P):
        d = O.unfold_digits(ranks, n, c)
        idx = [0 if k == n else int(d[k]) for k in range(len(ranks))]
        assert O.unfold_column(ranks, n, idx) == c
        seen.add(tuple(idx))
    assert len(seen) == P


# ---------------------------------------------------------------------------
# Model value x-hat
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape,ranks,R", [((4, 3, 5), (2, 3, 2), 2), ((3, 2, 4, 2), (2, 2, 3, 2), 3),
                                          ((5, 6), (3, 2), 4)])
def test_predict_equals_dense_bruteforce(shape, ranks, R):
    md = _random_model(shape, ranks, R, seed=11)
    G = _kruskal_core_numpy(md.B)
    X = _dense_reconstruction(G, md.A)
    coords = np.stack(np.unravel_index(np.arange(int(np.prod(shape))), shape), axis=1).astype(np.int32)
    got = md.predict(coords)
    want = X[tuple(coords.T)]
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)
    # the oracle's core equals the numpy Kruskal core
    np.testing.assert_allclose(md.core_tensor(), G, rtol=1e-13, atol=1e-13)


def test_predict_cp_identity():
    """A Kruskal core makes the model CP with factors A_n B_n:
    x-hat = sum_r prod_n (A_n B_n)[i_n, r]."""
    shape, ranks, R = (30, 20, 10, 5), (4, 3, 5, 2), 3
    md = _random_model(shape, ranks, R, seed=3)
    coords, _ = _random_batch(shape, 500, seed=4)
    C = [md.A[n] @ md.B[n] for n in range(4)]
    want = np.ones((500, R))
    for n in range(4):
        want *= C[n][coords[:, n]]
    np.testing.assert_allclose(md.predict(coords), want.sum(axis=1), rtol=1e-11, atol=1e-12)


def test_core_one_hot_columns():
    """Eq. 4 with one-hot Kruskal columns puts a 1 at each selected cell."""
    ranks, R = (3, 4, 2), 2
    B = [np.zeros((J, R)) for J in ranks]
    cells = [(2, 1, 0), (0, 3, 1)]
    for r, cell in enumerate(cells):
        for n in range(3):
            B[n][cell[n], r] = 1.0
    md = O.Model((5, 5, 5), ranks, R, [np.zeros((5, J)) for J in ranks], B)
    G = md.core_tensor()
    want = np.zeros(ranks)
    for cell in cells:
        want[cell] = 1.0
    assert np.array_equal(G, want)


# ---------------------------------------------------------------------------
# Gradients (Eq. 15, Eq. 18) against central finite differences of the loss
#   f = (1/(2m)) sum_s (x-hat_s - x_s)^2 + (lambda/2) ||block||^2
# which is quadratic in each block, so central differences are exact up to
# rounding.
# ---------------------------------------------------------------------------

def _loss(md, coords, x, lam, block):
    e = md.predict(coords) - x.astype(np.float64)
    return 0.5 * float(np.dot(e, e)) / coords.shape[0] + 0.5 * lam * float(np.dot(block, block))


@pytest.mark.parametrize("literal", [False, True])
@pytest.mark.parametrize("shape,ranks,R", [((6, 5, 4), (3, 2, 4), 3), ((4, 3, 3, 5), (2, 3, 2, 2), 2)])
def test_core_gradient_finite_differences(shape, ranks, R, literal):
    md = _random_model(shape, ranks, R, seed=21, scale=0.7)
    coords, x = _random_batch(shape, 17, seed=22)
    lam, h = 0.3, 1e-4
    for n in range(len(shape)):
        for r in range(R):
            g = md.core_gradient(coords, x, n, r, lam, literal=literal)
            fd = np.empty_like(g)
            for j in range(ranks[n]):
                b0 = md.B[n][j, r]
                md.B[n][j, r] = b0 + h
                fp = _loss(md, coords, x, lam, md.B[n][:, r])
                md.B[n][j, r] = b0 - h
                fm = _loss(md, coords, x, lam, md.B[n][:, r])
                md.B[n][j, r] = b0
                fd[j] = (fp - fm) / (2 * h)
            np.testing.assert_allclose(g, fd, rtol=1e-7, atol=1e-9)


@pytest.mark.parametrize("norm_mode", [0, 1])
@pytest.mark.parametrize("shape,ranks,R", [((6, 5, 4), (3, 2, 4), 3), ((4, 3, 3, 5), (2, 3, 2, 2), 2)])
def test_factor_gradient_finite_differences(shape, ranks, R, norm_mode):
    md = _random_model(shape, ranks, R, seed=31, scale=0.7)
    coords, x = _random_batch(shape, 23, seed=32, distinct=False)
    lam, h = 0.2, 1e-4
    m = coords.shape[0]
    for n in range(len(shape)):
        for row in np.unique(coords[:, n]):
            sel = coords[:, n] == row
            cnt = int(sel.sum())
            g = md.factor_gradient(coords, x, n, int(row), lam, norm_mode)
            fd = np.empty_like(g)
            for j in range(ranks[n]):
                a0 = md.A[n][row, j]
                md.A[n][row, j] = a0 + h
                fp = _loss(md, coords[sel], x[sel], lam, md.A[n][row])
                md.A[n][row, j] = a0 - h
                fm = _loss(md, coords[sel], x[sel], lam, md.A[n][row])
                md.A[n][row, j] = a0
                fd[j] = (fp - fm) / (2 * h)
            # _loss normalises by the row's own count; Eq. 18 by M (mode 0)
            denom = m if norm_mode == 0 else cnt
            data_fd = fd - lam * md.A[n][row]
            np.testing.assert_allclose(g - lam * md.A[n][row], data_fd * cnt / denom,
                                       rtol=1e-7, atol=1e-9)


def test_literal_and_closed_form_steps_agree():
    """W_r = H O_r (Algorithm 1, core phase, Eq. 7) equals the closed form."""
    shape, ranks, R = (5, 4, 6), (3, 2, 3), 2
    coords, x = _random_batch(shape, 19, seed=41, distinct=False)
    a = _random_model(shape, ranks, R, seed=42)
    b = a.copy()
    Va, Fa, Sa = a.step(coords, x, 0.05, 0.05, 0.01, 0.02, literal=False, probe=True)
    Vb, Fb, Sb = b.step(coords, x, 0.05, 0.05, 0.01, 0.02, literal=True, probe=True)
    np.testing.assert_allclose(Va, Vb, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(Fa, Fb, rtol=1e-12, atol=1e-12)
    assert np.array_equal(Sa, Sb)
    for n in range(3):
        np.testing.assert_allclose(a.A[n], b.A[n], rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(a.B[n], b.B[n], rtol=1e-12, atol=1e-13)


def test_step_probe_matches_gradient_functions():
    """The V recorded for (mode 1, r_core 1) of a step is the Eq. 15 bracket at
    the start of the step; the factor F of mode 1 uses the core after the core
    phase (Algorithm 1, Eq. 4)."""
    shape, ranks, R = (6, 5, 4), (3, 2, 4), 3
    coords, x = _random_batch(shape, 21, seed=43, distinct=False)
    md = _random_model(shape, ranks, R, seed=44)
    lam_b = 0.01
    g00 = md.core_gradient(coords, x, 0, 0, lam_b)
    V, F, S = md.copy().step(coords, x, 0.1, 0.1, 0.0, lam_b, probe=True)
    np.testing.assert_allclose(V[0, 0, :3] / coords.shape[0] + lam_b * md.B[0][:, 0], g00, rtol=1e-12)


# ---------------------------------------------------------------------------
# Whole step: the N=2, B(1)=B(2)=I special case is textbook alternating
# matrix-factorisation SGD on the rows u = a^(1)_i, v = a^(2)_k.
# ---------------------------------------------------------------------------

def test_matrix_factorisation_special_case():
    J = 3
    g = _rng(7)
    U = g.standard_normal((5, J))
    Vm = g.standard_normal((4, J))
    md = O.Model((5, 4), (J, J), J, [U, Vm], [np.eye(J), np.eye(J)])
    coords = np.array([[2, 1], [2, 3], [0, 1]], dtype=np.int32)
    x = np.array([0.7, -1.2, 0.4], dtype=np.float32)
    gam, lam = 0.3, 0.05
    md.step(coords, x, gam, 0.0, lam, 0.0)
    # textbook: for each user row, u <- u + gamma*(sum_k err_k v_k / M - lam u)
    M = 3
    u, v = U.copy(), Vm.copy()
    for i in np.unique(coords[:, 0]):
        grad = np.zeros(J)
        for s in np.where(coords[:, 0] == i)[0]:
            k = coords[s, 1]
            err = float(x[s]) - u[i] @ v[k]
            grad += err * v[k]
        u[i] = u[i] + gam * (grad / M - lam * u[i])
    v_new = v.copy()
    for k in np.unique(coords[:, 1]):
        grad = np.zeros(J)
        for s in np.where(coords[:, 1] == k)[0]:
            i = coords[s, 0]
            err = float(x[s]) - u[i] @ v[k]
            grad += err * u[i]
        v_new[k] = v[k] + gam * (grad / M - lam * v[k])
    np.testing.assert_allclose(md.A[0], u, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(md.A[1], v_new, rtol=1e-13, atol=1e-14)
    np.testing.assert_array_equal(md.B[0], np.eye(J))


def test_momentum_matrix_factorisation_two_steps():
    # Heavy-ball momentum on the N = 2, B = I case: textbook alternating
    # matrix-factorisation SGD with a velocity per row (v <- mu v + g,
    # w <- w - gamma v, g the regularised gradient), two minibatches.
    J, mu = 3, 0.7
    g = _rng(11)
    U = g.standard_normal((5, J))
    Vm = g.standard_normal((4, J))
    md = O.Model((5, 4), (J, J), J, [U, Vm], [np.eye(J), np.eye(J)], momentum=mu)
    batches = [(np.array([[2, 1], [2, 3], [0, 1]], dtype=np.int32), np.array([0.7, -1.2, 0.4], dtype=np.float32)),
               (np.array([[2, 0], [1, 1], [0, 1], [4, 3]], dtype=np.int32),
                np.array([0.1, 0.9, -0.5, 0.3], dtype=np.float32))]
    gam, lam = 0.3, 0.05
    u, v = U.copy(), Vm.copy()
    vu, vv = np.zeros_like(u), np.zeros_like(v)
    for coords, x in batches:
        md.step(coords, x, gam, 0.0, lam, 0.0)
        M = coords.shape[0]
        for i in np.unique(coords[:, 0]):
            grad = np.zeros(J)
            for s in np.where(coords[:, 0] == i)[0]:
                k = coords[s, 1]
                grad += (u[i] @ v[k] - float(x[s])) * v[k]
            vu[i] = mu * vu[i] + (grad / M + lam * u[i])
            u[i] = u[i] - gam * vu[i]
        v_new = v.copy()
        for k in np.unique(coords[:, 1]):
            grad = np.zeros(J)
            for s in np.where(coords[:, 1] == k)[0]:
                i = coords[s, 0]
                grad += (u[i] @ v[k] - float(x[s])) * u[i]
            vv[k] = mu * vv[k] + (grad / M + lam * v[k])
            v_new[k] = v[k] - gam * vv[k]
        v = v_new
    np.testing.assert_allclose(md.A[0], u, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(md.A[1], v, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(md.VA[0], vu, rtol=1e-13, atol=1e-14)


def test_momentum_first_step_is_plain_sgd_and_zero_momentum_is_sgd():
    # The velocity starts at zero, so the first step with any mu is the plain
    # step; with mu = 0 every step is the plain step.
    shape, ranks, R = (8, 7, 6), (3, 2, 3), 2
    coords, x = _random_batch(shape, 40, seed=57)
    base = _random_model(shape, ranks, R, seed=58, scale=0.5)
    plain = O.Model(shape, ranks, R, base.A, base.B)
    mom = O.Model(shape, ranks, R, base.A, base.B, momentum=0.9)
    zero = O.Model(shape, ranks, R, base.A, base.B, momentum=0.0)
    for md in (plain, mom, zero):
        md.step(coords, x, 0.1, 0.05, 0.01, 0.02)
    for n in range(3):
        np.testing.assert_array_equal(mom.A[n], plain.A[n])
        np.testing.assert_array_equal(mom.B[n], plain.B[n])
    coords2, x2 = _random_batch(shape, 40, seed=59)
    for md in (plain, mom, zero):
        md.step(coords2, x2, 0.1, 0.05, 0.01, 0.02)
    for n in range(3):
        np.testing.assert_array_equal(zero.A[n], plain.A[n])
        assert not np.array_equal(mom.A[n], plain.A[n])


def test_momentum_kruskal_columns_three_steps_by_hand():
    # Heavy-ball on the Kruskal columns alone (lr_a = 0 freezes every factor
    # row), written out from the model's definition: x-hat_s = sum_r prod_n
    # <a(n)_{i_n}, b(n)_r> (Def. 6 with the core of Eq. 4), so the bracket of
    # Eq. 15 for column r of mode n is V = sum_s (x-hat_s - x_s) w_s[r] a(n)_{i_n},
    # w_s[r] = prod_{k != n} <a(k)_{i_k}, b(k)_r>, with x-hat taken at the
    # current columns (Algorithm 1 moves one column at a time, modes in order).
    # Then g = V / M + lambda b, v <- mu v + g, b <- b - gamma v, velocities
    # carried from one minibatch to the next.  A velocity that is not carried,
    # or one kept under the wrong (mode, j, r) index, changes steps 2 and 3.
    shape, ranks, R, mu = (6, 5, 4), (3, 2, 3), 3, 0.6
    gam, lam = 0.05, 0.02
    base = _random_model(shape, ranks, R, seed=61, scale=0.7)
    md = O.Model(shape, ranks, R, base.A, base.B, momentum=mu)
    A = [a.copy() for a in base.A]
    Bh = [b.copy() for b in base.B]
    VB = [np.zeros_like(b) for b in Bh]
    for step in range(3):
        coords, x = _random_batch(shape, 15, seed=70 + step, distinct=False)
        md.step(coords, x, 0.0, gam, 0.3, lam)
        M = coords.shape[0]
        rows = [A[n][coords[:, n]] for n in range(3)]          # a(n)_{i_n} per sample, M x J_n
        for n in range(3):
            for r in range(R):
                dots = np.stack([rows[k] @ Bh[k] for k in range(3)])     # [k][s][r']
                xhat = np.prod(dots, axis=0).sum(axis=1)
                w = np.prod([dots[k][:, r] for k in range(3) if k != n], axis=0)
                V = ((xhat - x.astype(np.float64)) * w) @ rows[n]
                g = V / M + lam * Bh[n][:, r]
                VB[n][:, r] = mu * VB[n][:, r] + g
                Bh[n][:, r] = Bh[n][:, r] - gam * VB[n][:, r]
        for n in range(3):
            np.testing.assert_allclose(md.B[n], Bh[n], rtol=1e-11, atol=1e-13)
            np.testing.assert_allclose(md.VB[n], VB[n], rtol=1e-11, atol=1e-13)
            np.testing.assert_array_equal(md.A[n], A[n])


# ---------------------------------------------------------------------------
# Descent (Theorem 3): each block step is a small gradient step on a convex
# quadratic, so the sampled objective decreases.
# ---------------------------------------------------------------------------

def test_step_decreases_sampled_objective():
    shape, ranks, R = (8, 7, 6), (3, 3, 3), 2
    coords, x = _random_batch(shape, 64, seed=51)
    md = _random_model(shape, ranks, R, seed=52, scale=0.6)
    lam = 0.01

    def objective(m):
        e = m.predict(coords) - x
        reg = sum(float(np.sum(b * b)) for b in m.B)
        for n in range(3):
            rows = np.unique(coords[:, n])
            reg += float(np.sum(m.A[n][rows] ** 2))
        return 0.5 * float(e @ e) / 64 + 0.5 * lam * reg

    prev = objective(md)
    for _ in range(5):
        md.step(coords, x, 0.05, 0.05, lam, lam)
        cur = objective(md)
        assert cur < prev
        prev = cur


# ---------------------------------------------------------------------------
# Sampler and tiler
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 8, 9, 100, 1023, 1024, 1025, 4097, 65536, 65537, 200003])
def test_sampler_is_a_permutation(n):
    p = O.epoch_schedule(n, seed=2, epoch=3)
    assert p.shape == (n,)
    assert np.array_equal(np.sort(p), np.arange(n))


def test_sampler_depends_on_seed_and_epoch():
    n = 10007
    a = O.epoch_schedule(n, 2, 0)
    b = O.epoch_schedule(n, 2, 1)
    c = O.epoch_schedule(n, 3, 0)
    assert np.array_equal(a, O.epoch_schedule(n, 2, 0))
    assert (a != b).mean() > 0.99 and (a != c).mean() > 0.99
    assert O.perm(n, 2, 1, 17) == b[17]


def test_sampler_positions_are_uniform():
    """Where entry 0 lands over many epochs is uniform over [0, n) (chi-square)."""
    n, epochs = 64, 6400
    hits = np.zeros(n)
    for e in range(epochs):
        p = O.epoch_schedule(n, 9, e)
        hits[int(np.where(p == 0)[0][0])] += 1
    exp = epochs / n
    chi2 = float(((hits - exp) ** 2 / exp).sum())
    assert chi2 < 120.0          # 63 dof: P(chi2 > 120) ~ 1e-5
    # consecutive positions are not correlated with the identity
    p = O.epoch_schedule(100000, 1, 0)
    assert abs(np.corrcoef(np.arange(100000), p)[0, 1]) < 0.02


@pytest.mark.parametrize("m,hi", [(1, 5), (17, 3), (256, 50), (4096, 500000), (3000, 1)])
def test_stable_order_matches_library_stable_sort(m, hi):
    keys = _rng(m).integers(0, hi, size=m).astype(np.int32)
    order, seg = O.stable_order(keys)
    assert np.array_equal(order, np.argsort(keys, kind="stable"))
    uniq, first = np.unique(keys, return_index=True)
    starts = np.searchsorted(keys[order], uniq, side="left")
    assert np.array_equal(seg[:-1], starts) and seg[-1] == m


# ---------------------------------------------------------------------------
# RMSE / MAE (Eq. 19) on residual patterns with closed-form answers.
# ---------------------------------------------------------------------------

def test_rmse_mae_closed_form():
    shape, ranks = (4, 4, 4), (2, 2, 2)
    md = O.Model(shape, ranks, 1, [np.zeros((4, 2))] * 3, [np.ones((2, 1))] * 3)
    coords = np.array([[0, 0, 0], [1, 2, 3]], dtype=np.int32)
    r, a = md.rmse_mae(coords, np.array([3.0, -4.0], dtype=np.float32))
    assert r == pytest.approx(math.sqrt(12.5), rel=1e-15)
    assert a == pytest.approx(3.5, rel=1e-15)
    # an exact model has zero error
    md2 = _random_model(shape, ranks, 2, seed=5)
    c, _ = _random_batch(shape, 30, seed=6)
    vals = md2.predict(c)
    r2, a2 = md2.rmse_mae(c, vals.astype(np.float32))
    assert r2 < 1e-6 and a2 < 1e-6


# ---------------------------------------------------------------------------
# Epoch driver: minibatch b is pi_e([bM, bM+M)) and the last batch is ragged.
# ---------------------------------------------------------------------------

def test_epoch_equals_manual_minibatches():
    shape, ranks, R = (9, 8, 7), (3, 2, 3), 2
    coords, x = _random_batch(shape, 103, seed=61)
    M, seed, ep = 16, 2, 4
    a = _random_model(shape, ranks, R, seed=62)
    b = a.copy()
    a.epoch(coords, x, M, seed, ep, 0.05, 0.04, 0.01, 0.02)
    sched = O.epoch_schedule(103, seed, ep)
    for t0 in range(0, 103, M):
        ids = sched[t0:t0 + M]
        b.step(coords[ids], x[ids], 0.05, 0.04, 0.01, 0.02)
    for n in range(3):
        np.testing.assert_array_equal(a.A[n], b.A[n])
        np.testing.assert_array_equal(a.B[n], b.B[n])


# ---------------------------------------------------------------------------
# Iteration as a whole: recover a planted, exactly representable model
# (Kruskal core, J=4, R=3) from half of a 30x30x30 tensor with N(0, 0.01^2)
# noise; the held-out RMSE must reach the noise floor (<= 2 sigma).
# ---------------------------------------------------------------------------

def test_planted_kruskal_core_recovery():
    g = np.random.default_rng(0)
    shape, ranks, R, sigma = (30, 30, 30), (4, 4, 4), 3, 0.01
    truth = O.Model(shape, ranks, R, [g.standard_normal((30, 4)) / 2 for _ in range(3)],
                    [g.standard_normal((4, R)) for _ in range(3)])
    lin = g.choice(27000, size=13500, replace=False)
    coords = np.stack(np.unravel_index(lin, shape), axis=1).astype(np.int32)
    x = (truth.predict(coords) + sigma * g.standard_normal(13500)).astype(np.float32)
    tr, te = slice(0, 12150), slice(12150, 13500)
    g2 = np.random.default_rng(5)
    md = O.Model(shape, ranks, R, [0.3 * g2.standard_normal((30, 4)) for _ in range(3)],
                 [g2.standard_normal((4, R)) for _ in range(3)])
    start = md.rmse_mae(coords[te], x[te])[0]
    for ep in range(150):
        md.epoch(coords[tr], x[tr], 1, 2, ep, 0.002, 0.002, 1e-4, 1e-4)
    end = md.rmse_mae(coords[te], x[te])[0]
    assert start > 50 * sigma
    assert end <= 2 * sigma


@pytest.mark.parametrize("norm_mode", [0, 1])
def test_step_is_cyclic_block_sgd(norm_mode):
    """Algorithm 1 order: for n = 1..N, r = 1..R, b^(n)_r takes an SGD step on
    its Eq. 15 gradient at the current state (Gauss-Seidel across r and n);
    then for n = 1..N every touched row of A(n) takes an SGD step on its
    Eq. 18 gradient at the state after modes < n (rows of one mode jointly).
    Rebuilt here from the finite-difference-pinned gradient functions."""
    shape, ranks, R = (7, 6, 5), (3, 2, 3), 3
    coords, x = _random_batch(shape, 29, seed=71, distinct=False)
    md = _random_model(shape, ranks, R, seed=72, scale=0.8)
    ref = md.copy()
    ga, gb, la, lb = 0.07, 0.05, 0.02, 0.03
    V, F, nseg = md.step(coords, x, ga, gb, la, lb, norm_mode=norm_mode, probe=True)
    m = coords.shape[0]
    for n in range(3):
        for r in range(R):
            g = ref.core_gradient(coords, x, n, r, lb)
            np.testing.assert_allclose(V[n, r, :ranks[n]] / m + lb * ref.B[n][:, r], g, rtol=1e-12, atol=1e-13)
            ref.B[n][:, r] = ref.B[n][:, r] - gb * g
    for n in range(3):
        rows = np.unique(coords[:, n])
        assert nseg[n] == rows.size
        grads = [ref.factor_gradient(coords, x, n, int(i), la, norm_mode) for i in rows]
        for i, g in zip(rows, grads):
            ref.A[n][i] = ref.A[n][i] - ga * g
    for n in range(3):
        np.testing.assert_allclose(md.B[n], ref.B[n], rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(md.A[n], ref.A[n], rtol=1e-12, atol=1e-13)


# ---------------------------------------------------------------------------
# K-snapshot form (a labelled variant of the minibatch order): blocks of K
# minibatches, each stepping from the block's starting model; their changes
# are added to it in minibatch order.
# ---------------------------------------------------------------------------

def test_snapshot_k1_is_the_strict_sequence_bit_for_bit():
    shape, ranks, R = (9, 8, 7), (3, 2, 3), 2
    coords, x = _random_batch(shape, 150, seed=81)
    base = _random_model(shape, ranks, R, seed=82, scale=0.6)
    strict = O.Model(shape, ranks, R, base.A, base.B)
    snap = O.Model(shape, ranks, R, base.A, base.B)
    strict.epoch(coords, x, 16, 5, 0, 0.2, 0.1, 0.01, 0.02)
    snap.epoch_snapshot(coords, x, 16, 5, 0, 1, 0.2, 0.1, 0.01, 0.02)
    for n in range(3):
        np.testing.assert_array_equal(snap.A[n], strict.A[n])
        np.testing.assert_array_equal(snap.B[n], strict.B[n])


def _mf_step_delta(U, Vm, coords, x, gam, lam):
    """One minibatch of textbook alternating matrix-factorisation SGD from
    (U, Vm): the changes it makes to the rows of U, then (with U updated) to
    the rows of Vm, as dicts row -> change."""
    M = coords.shape[0]
    dU, dV = {}, {}
    U1 = U.copy()
    for i in np.unique(coords[:, 0]):
        grad = np.zeros(U.shape[1])
        for s in np.where(coords[:, 0] == i)[0]:
            grad += (U[i] @ Vm[coords[s, 1]] - float(x[s])) * Vm[coords[s, 1]]
        dU[i] = -(gam * (grad / M + lam * U[i]))
        U1[i] = U[i] + dU[i]
    for k in np.unique(coords[:, 1]):
        grad = np.zeros(U.shape[1])
        for s in np.where(coords[:, 1] == k)[0]:
            grad += (U1[coords[s, 0]] @ Vm[k] - float(x[s])) * U1[coords[s, 0]]
        dV[k] = -(gam * (grad / M + lam * Vm[k]))
    return dU, dV


def test_snapshot_k2_matrix_factorisation_by_hand():
    # N = 2, B = I, lr_b = 0: the factor phase is textbook alternating MF SGD.
    # Two blocks of K = 2 minibatches (the second block a single short one):
    # in a block both minibatches step from the block's start, and the rows'
    # changes are added in minibatch order (row 2 is touched by both).
    J = 3
    g = _rng(83)
    U = g.standard_normal((5, J))
    Vm = g.standard_normal((4, J))
    md = O.Model((5, 4), (J, J), J, [U, Vm], [np.eye(J), np.eye(J)])
    coords = np.array([[2, 1], [2, 3], [0, 1], [2, 0], [1, 1], [4, 3], [3, 2]], dtype=np.int32)
    x = np.array([0.7, -1.2, 0.4, 0.1, 0.9, -0.5, 0.3], dtype=np.float32)
    gam, lam, M, K = 0.3, 0.05, 3, 2
    # the oracle's minibatch b holds the entries at positions pi_0(bM ..)
    order = O.perm_range(7, 2, 0, 0, 7)
    md.epoch_snapshot(coords[order], x[order], M, 2, 0, K, gam, 0.0, lam, 0.0)
    # by hand: re-read the same permutation of the permuted arrays
    perm = O.perm_range(7, 2, 0, 0, 7)
    cb, xb = coords[order][perm], x[order][perm]
    u, v = U.copy(), Vm.copy()
    for q0 in range(0, 3, K):
        u0, v0 = u.copy(), v.copy()
        for b in range(q0, min(q0 + K, 3)):
            sl = slice(b * M, min((b + 1) * M, 7))
            dU, dV = _mf_step_delta(u0, v0, cb[sl], xb[sl], gam, lam)
            for i, d in dU.items():
                u[i] = u[i] + d
            for k, d in dV.items():
                v[k] = v[k] + d
    np.testing.assert_allclose(md.A[0], u, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(md.A[1], v, rtol=1e-13, atol=1e-14)
    np.testing.assert_array_equal(md.B[0], np.eye(J))


def test_snapshot_k2_kruskal_columns_by_hand():
    # lr_a = 0: only the core phase moves.  Each minibatch of the block runs
    # the cyclic column updates (Eq. 15 bracket from the model's definition)
    # from the block's starting B; the column changes are added in order.
    shape, ranks, R = (6, 5, 4), (3, 2, 3), 3
    gam, lam, M, K = 0.05, 0.02, 12, 2
    base = _random_model(shape, ranks, R, seed=84, scale=0.7)
    coords, x = _random_batch(shape, 36, seed=85, distinct=False)
    md = O.Model(shape, ranks, R, base.A, base.B)
    md.epoch_snapshot(coords, x, M, 3, 1, K, 0.0, gam, 0.4, lam)
    perm = O.perm_range(36, 3, 1, 0, 36)
    cb, xb = coords[perm], x[perm].astype(np.float64)
    A = [a.copy() for a in base.A]
    Bh = [b.copy() for b in base.B]
    for q0 in range(0, 3, K):
        B0 = [b.copy() for b in Bh]
        for b in range(q0, min(q0 + K, 3)):
            sl = slice(b * M, (b + 1) * M)
            rows = [A[n][cb[sl, n]] for n in range(3)]
            W = [b_.copy() for b_ in B0]
            for n in range(3):
                for r in range(R):
                    dots = np.stack([rows[k] @ W[k] for k in range(3)])
                    xhat = np.prod(dots, axis=0).sum(axis=1)
                    w = np.prod([dots[k][:, r] for k in range(3) if k != n], axis=0)
                    V = ((xhat - xb[sl]) * w) @ rows[n]
                    d = -(gam * (V / M + lam * W[n][:, r]))
                    W[n][:, r] = W[n][:, r] + d
                    Bh[n][:, r] = Bh[n][:, r] + d
    for n in range(3):
        np.testing.assert_allclose(md.B[n], Bh[n], rtol=1e-11, atol=1e-13)
        np.testing.assert_array_equal(md.A[n], A[n])


def test_snapshot_block_covering_the_epoch_steps_everything_from_the_start():
    # K at least the number of minibatches: every minibatch steps from the
    # initial model, so the result is the initial model plus the sum of the
    # single-minibatch changes, whatever their order of computation.
    shape, ranks, R = (7, 6, 5), (2, 3, 2), 2
    coords, x = _random_batch(shape, 40, seed=86)
    base = _random_model(shape, ranks, R, seed=87, scale=0.6)
    md = O.Model(shape, ranks, R, base.A, base.B)
    md.epoch_snapshot(coords, x, 10, 4, 2, 8, 0.2, 0.1, 0.01, 0.02)
    perm = O.perm_range(40, 4, 2, 0, 40)
    want_A = [a.copy() for a in base.A]
    want_B = [b.copy() for b in base.B]
    for b in range(4):
        one = O.Model(shape, ranks, R, base.A, base.B)
        sl = perm[b * 10:(b + 1) * 10]
        one.step(coords[sl], x[sl], 0.2, 0.1, 0.01, 0.02)
        for n in range(3):
            want_A[n] += one.A[n] - base.A[n]
            want_B[n] += one.B[n] - base.B[n]
    for n in range(3):
        np.testing.assert_allclose(md.A[n], want_A[n], rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(md.B[n], want_B[n], rtol=1e-12, atol=1e-14)
