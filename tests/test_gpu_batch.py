"""Batched epochs (many independent decompositions in one persistent launch).

Each tensor of a batch must get exactly the epoch std_sgd_epoch gives it on
its own with the same number of CTAs (bit for bit: same code, same chunking,
fixed summation orders), whatever the other tensors in the launch; the
group-size tuner must leave every parameter untouched; and one member is
checked against the FP64 oracle.
"""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import __graft_entry__ as ge
    ge.build()
    from paper_2012_03550_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def synth():
    from paper_2012_03550_gb300 import synth as s
    return s


# uneven members: orders 3 and 4, J in {4, 8, 16}, 1.5K..30K nonzeros, one
# Zipf-skewed tensor whose hot rows span several chunks
SPECS = [
    ((300, 200, 100), 30000, (8, 8, 8), 5, [("zipf", 1.2), ("zipf", 1.2), ("uniform",)]),
    ((120, 90, 60), 6000, (4, 4, 4), 4, [("uniform",)] * 3),
    ((80, 70, 60, 12), 9000, (4, 4, 4, 4), 3, [("uniform",)] * 4),
    ((500, 40, 30), 1500, (16, 16, 16), 5, [("uniform",)] * 3),
    ((200, 150, 90), 12000, (8, 4, 16), 5, [("zipf", 1.1), ("uniform",), ("uniform",)]),
    ((60, 50, 40), 2500, (4, 8, 4), 2, [("uniform",)] * 3),
]


def _members(B, synth, ctas=0, **opts):
    out = []
    for k, (shape, nnz, ranks, R, dists) in enumerate(SPECS):
        t = synth.make_tensor(shape, nnz, dists, ranks, 0.05, 0.1, seed=100 + k)
        c, v = t.split("train")
        A0, B0 = synth.init_params(shape, ranks, R, mode="normal", seed=1)
        g = B.Tucker(shape, ranks, c, v, r_core=R, ctas=ctas, **opts)
        g.set_params(A0, B0, epoch=0)
        out.append((t, g, A0, B0, ranks, R))
    return out


def _params_equal(ga, gb):
    Aa, Ba, ca, ea = ga.get_params()
    Ab, Bb, cb, eb = gb.get_params()
    return ea == eb and all(np.array_equal(x, y) for x, y in zip(Aa, Ab)) and \
        all(np.array_equal(x, y) for x, y in zip(Ba, Bb)) and np.array_equal(ca, cb)


@pytest.mark.parametrize("group,opts", [(4, {}), (2, {"contraction": 1}), (4, {"momentum": 0.5})])
def test_batch_equals_each_tensor_alone(B, synth, group, opts):
    M, lr, lam = 256, 0.1, 1e-3
    batched = _members(B, synth, **opts)
    alone = _members(B, synth, ctas=group, **opts)
    with B.Batch([m[1] for m in batched], ctas_per_tensor=group) as bt:
        for _ in range(2):
            st = bt.epoch(lr, lr, lam, lam, M)
            assert st["ctas_per_tensor"] == group and st["tensors"] == len(SPECS)
    for m in alone:
        for _ in range(2):
            m[1].epoch(lr, lr, lam, lam, M)
    for a, b in zip(batched, alone):
        assert _params_equal(a[1], b[1])
    for m in batched + alone:
        m[1].close()


def test_batch_tuner_writes_nothing_and_matches_alone(B, synth):
    """Tuned base size plus larger groups for the long tensors: each tensor
    equals its run alone with the CTAs it was given."""
    M, lr, lam = 256, 0.1, 1e-3
    batched = _members(B, synth)
    with B.Batch([m[1] for m in batched], ctas_per_tensor=0) as bt:
        st = bt.epoch(lr, lr, lam, lam, M)
        group = st["ctas_per_tensor"]
        sizes = bt.groups()
        tile = bt.tile()
    assert tile in (0, 1, 2, 4)   # the contraction tile the tuner kept (same bits whatever it is)
    assert group >= 1 and len(sizes) == len(SPECS)
    assert all(g >= group and g % group == 0 for g in sizes)
    for k, (a, g) in enumerate(zip(batched, sizes)):
        shape, nnz, ranks, R, dists = SPECS[k]
        t, _, A0, B0, _, _ = a
        c, v = t.split("train")
        alone = B.Tucker(shape, ranks, c, v, r_core=R, ctas=g)
        alone.set_params(A0, B0, epoch=0)
        alone.epoch(lr, lr, lam, lam, M)
        assert _params_equal(a[1], alone)
        alone.close()
    for m in batched:
        m[1].close()


def test_batch_long_tensor_gets_a_larger_group(B, synth):
    """One tensor far longer than the rest is promoted to a group of 2^k x the
    base size, and still equals its run alone with that many CTAs."""
    M, lr, lam = 256, 0.1, 1e-3
    specs = [((400, 300, 200), 60000, (8, 8, 8), 5, [("uniform",)] * 3)] + \
            [((60, 50, 40), 1500, (4, 4, 4), 3, [("uniform",)] * 3)] * 12
    mem = []
    for k, (shape, nnz, ranks, R, dists) in enumerate(specs):
        t = synth.make_tensor(shape, nnz, dists, ranks, 0.05, 0.1, seed=500 + k)
        c, v = t.split("train")
        A0, B0 = synth.init_params(shape, ranks, R, mode="normal", seed=1)
        g = B.Tucker(shape, ranks, c, v, r_core=R)
        g.set_params(A0, B0, epoch=0)
        mem.append((t, g, A0, B0, shape, ranks, R))
    with B.Batch([m[1] for m in mem], ctas_per_tensor=0) as bt:
        st = bt.epoch(lr, lr, lam, lam, M)
        sizes = bt.groups()
    base = st["ctas_per_tensor"]
    assert sizes[0] == max(sizes) and (sizes[0] > base or base == 32), (sizes, base)
    assert all(n == base for n in sizes[1:])
    for (t, g, A0, B0, shape, ranks, R), n in zip(mem, sizes):
        c, v = t.split("train")
        alone = B.Tucker(shape, ranks, c, v, r_core=R, ctas=n)
        alone.set_params(A0, B0, epoch=0)
        alone.epoch(lr, lr, lam, lam, M)
        assert _params_equal(g, alone)
        alone.close()
        g.close()


def test_batch_member_tracks_oracle(B, synth):
    M, lr, lam = 256, 0.1, 1e-3
    batched = _members(B, synth)
    t, g, A0, B0, ranks, R = batched[0]
    c, v = t.split("train")
    tc, tv = t.split("test")
    ref = O.Model(t.shape, ranks, R, A0, B0)
    worst = 0.0
    with B.Batch([m[1] for m in batched], ctas_per_tensor=4) as bt:
        for ep in range(3):
            bt.epoch(lr, lr, lam, lam, M)
            ref.epoch(c, v, M, 2, ep, lr, lr, lam, lam)
            r_g, m_g = g.rmse(tc, tv)
            r_o, m_o = ref.rmse_mae(tc, tv)
            worst = max(worst, abs(r_g - r_o), abs(m_g - m_o))
    assert worst <= 1e-3, worst
    for m in batched:
        m[1].close()


@pytest.mark.parametrize("group", [2, 4, 8, 16])
def test_cluster_form_equals_cooperative_form(B, synth, group):
    """A group of 2..16 CTAs runs as one thread block cluster (exchanges through
    cluster barriers and shared memory); the cooperative form (tagged words
    through L2) runs when any group of the launch is larger.  Both add the
    same numbers in the same order, so they agree bit for bit: members at
    `group` CTAs beside one 32-CTA group (cooperative form) against their runs
    alone at `group` CTAs (cluster form)."""
    M, lr, lam = 256, 0.1, 1e-3
    batched = _members(B, synth)
    alone = _members(B, synth, ctas=group)
    sizes = [group] * (len(SPECS) - 1) + [32]
    with B.Batch([m[1] for m in batched], ctas_per_tensor=group) as bt:
        bt.set_groups(sizes)
        for _ in range(2):
            bt.epoch(lr, lr, lam, lam, M)
        assert bt.groups() == sizes
    for m in alone[:-1]:
        for _ in range(2):
            m[1].epoch(lr, lr, lam, lam, M)
    for a, b in zip(batched[:-1], alone[:-1]):
        assert _params_equal(a[1], b[1])
    for m in batched + alone:
        m[1].close()
