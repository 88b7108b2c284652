"""Pins of the oracle's n-body and particle-collision workloads (Table 1 "nbody",
"collision"; the n-body listing of Sec. 2).

The paper prints no numbers for these applications, so the oracle is pinned by
physics that does not depend on the code: free motion, the first step of a pair
at rest and the circular two-body orbit (Kepler), Newton's third law (exact here
because of the fixed-point force sums), momentum and mass conservation, merges
derived by hand for two and three bodies, and independence of the visit order.
"""
import math

import numpy as np
import pytest

import oracle

S = 2.0 ** 40


def run(init, steps, **kw):
    init = np.asarray(init, np.float32)
    kw.setdefault("fscale", S)
    kw.setdefault("eps2", 2.0 ** -40)
    kw.setdefault("dt", 2.0 ** -4)
    return oracle.nbody_run(init.shape[0], steps, init=init, **kw)


def test_lone_body_moves_in_a_straight_line():
    st, alive, counts, fs = run([[0.125, -0.5, 0.001, -0.002, 3.0]], 50, G=2.0 ** -10)
    assert st[0, 2] == np.float32(0.001) and st[0, 3] == np.float32(-0.002)
    assert st[0, 4] == 3.0
    t = 50 * 2.0 ** -4
    assert abs(st[0, 0] - (0.125 + 0.001 * t)) < 1e-6
    assert abs(st[0, 1] - (-0.5 - 0.002 * t)) < 1e-6
    assert counts.tolist() == [1] * 51 and np.all(fs == 0)


def test_pair_at_rest_first_step_closed_form():
    G, a, m, dt, eps2 = 2.0 ** -10, 0.25, 2.0, 2.0 ** -4, 2.0 ** -6
    st, _, _, fs = run([[-a, 0, 0, 0, m], [a, 0, 0, 0, m]], 1, G=G, dt=dt, eps2=eps2)
    d2 = (2 * a) ** 2 + eps2
    F = G * m * m * (2 * a) / d2 ** 1.5          # attraction along +x for body 0
    v = F / m * dt
    assert st[0, 2] == pytest.approx(v, rel=1e-5)
    assert st[0, 0] == pytest.approx(-a + v * dt, abs=1e-7)
    assert st[1, 2] == -st[0, 2] and st[1, 0] == -st[0, 0]       # exact symmetry
    assert st[0, 1] == 0 and st[0, 3] == 0
    assert fs.tolist() == [[0, 0]]


def test_unequal_masses_accelerate_inversely_to_mass():
    G, a, dt = 2.0 ** -10, 0.25, 2.0 ** -4
    st, _, _, _ = run([[-a, 0, 0, 0, 1.0], [a, 0, 0, 0, 3.0]], 1, G=G, dt=dt)
    assert st[0, 2] > 0 > st[1, 2]
    assert st[0, 2] == pytest.approx(-3.0 * st[1, 2], rel=1e-6)
    p = 1.0 * float(st[0, 2]) + 3.0 * float(st[1, 2])
    assert abs(p) <= 1e-6 * abs(float(st[0, 2]))


def test_circular_two_body_orbit_quarter_period():
    # equal masses m at distance 2r circle their centre with v^2 = G m / (4 r)
    G, r, m, dt = 2.0 ** -10, 0.25, 1.0, 2.0 ** -8
    v = math.sqrt(G * m / (4 * r))              # = 2^-5 exactly
    w = v / r
    steps = round((math.pi / 2) / w / dt)
    st, _, _, _ = run([[r, 0, 0, v, m], [-r, 0, 0, -v, m]], steps, G=G, dt=dt)
    t = steps * dt
    expect = np.array([r * math.cos(w * t), r * math.sin(w * t)])
    assert np.abs(st[0, :2] - expect).max() < 0.01 * r
    assert np.abs(st[1, :2] + expect).max() < 0.01 * r
    assert abs(math.hypot(*st[0, :2]) - r) < 0.01 * r
    assert abs(math.hypot(*st[0, 2:4]) - v) < 0.01 * v


@pytest.mark.parametrize("collide", [False, True])
def test_newton_third_law_is_exact(collide):
    _, _, _, fs = oracle.nbody_run(300, 6, 11, G=2.0 ** -20, dt=0.25, eps2=2.0 ** -18,
                                   rc2=2.0 ** -12, collide=collide)
    assert np.all(fs == 0)


def test_momentum_conserved_by_gravity():
    kw = dict(G=2.0 ** -24, dt=0.25, eps2=2.0 ** -18)
    s0, _, _, _ = oracle.nbody_run(400, 0, 5, **kw)
    s1, _, _, _ = oracle.nbody_run(400, 10, 5, **kw)
    p0 = (s0[:, 4:5].astype(np.float64) * s0[:, 2:4]).sum(0)
    p1 = (s1[:, 4:5].astype(np.float64) * s1[:, 2:4]).sum(0)
    scale = (s1[:, 4:5].astype(np.float64) * np.abs(s1[:, 2:4])).sum()
    assert np.abs(p1 - p0).max() <= 1e-5 * scale
    assert np.abs(s1[:, 2:4] - s0[:, 2:4]).max() > 0          # forces did act


RC2 = 2.0 ** -10
RC = math.sqrt(RC2)


def test_two_bodies_merge_inelastically():
    init = [[0.0, 0.0, 1e-3, 0.0, 2.0], [0.5 * RC, 0.0, -1e-3, 0.0, 1.0]]
    dt = 2.0 ** -4
    st, alive, counts, _ = run(init, 1, G=0.0, dt=dt, rc2=RC2, collide=True)
    assert counts.tolist() == [2, 1] and alive.tolist() == [1, 0]
    x0, x1 = 1e-3 * dt, 0.5 * RC - 1e-3 * dt                   # after the move
    assert st[0, 4] == 3.0
    assert st[0, 2] == pytest.approx((2 * 1e-3 - 1e-3) / 3, rel=1e-6)
    assert st[0, 0] == pytest.approx((2 * x0 + x1) / 3, rel=1e-6)
    assert st[1].tolist() == [0, 0, 0, 0, 0]


def test_equal_masses_lower_id_absorbs():
    init = [[0.0, 0.0, 0.0, 0.0, 4.0], [0.0, 0.5 * RC, 0.0, 0.0, 4.0]]
    st, alive, counts, _ = run(init, 2, G=0.0, rc2=RC2, collide=True)
    assert alive.tolist() == [1, 0] and counts.tolist() == [2, 1, 1]
    assert st[0, 4] == 8.0 and st[0, 1] == pytest.approx(0.25 * RC, rel=1e-6)


def test_merge_chain_resolves_one_link_per_step():
    # A(m1) - B(m2) - C(m3) on a line: A -> B and B -> C are within reach, A - C is
    # not.  Step 1: B is merging into C, so A waits; C absorbs B and moves to the
    # centre of mass (2*0.8 + 3*1.1)/5 = 0.98 rc, within reach of A.  Step 2: A
    # merges into C.
    init = [[0.0, 0, 0, 0, 1.0], [0.8 * RC, 0, 0, 0, 2.0], [1.1 * RC, 0, 0, 0, 3.0]]
    st, alive, counts, _ = run(init, 2, G=0.0, rc2=RC2, collide=True)
    assert counts.tolist() == [3, 2, 1]
    assert alive.tolist() == [0, 0, 1]
    assert st[2, 4] == 6.0
    assert st[2, 0] == pytest.approx(5 * 0.98 * RC / 6, rel=1e-5)
    st1, alive1, _, _ = run(init, 1, G=0.0, rc2=RC2, collide=True)
    assert alive1.tolist() == [1, 0, 1] and st1[2, 4] == 5.0
    assert st1[2, 0] == pytest.approx(0.98 * RC, rel=1e-5)


def test_two_proposers_lowest_id_first():
    # A and B both reach C but not each other: C takes A (lower id) at step 1 and B
    # at step 2.
    init = [[-0.5 * RC, 0, 0, 0, 1.0], [0.5 * RC, 0, 0, 0, 1.0], [0.0, 0, 0, 0, 5.0]]
    st1, alive1, _, _ = run(init, 1, G=0.0, rc2=RC2, collide=True)
    assert alive1.tolist() == [0, 1, 1]
    assert st1[2, 0] == pytest.approx(-0.5 * RC / 6, rel=1e-5)
    st, alive, counts, _ = run(init, 2, G=0.0, rc2=RC2, collide=True)
    assert counts.tolist() == [3, 2, 1] and alive.tolist() == [0, 0, 1]
    assert st[2, 4] == 7.0 and st[2, 0] == pytest.approx(0.0, abs=1e-7)


def test_far_bodies_never_merge():
    xs = np.arange(6, dtype=np.float32) * np.float32(2 * RC)
    init = np.stack([xs, np.zeros(6), np.zeros(6), np.zeros(6), np.arange(1, 7)], 1)
    st, alive, counts, _ = run(init, 5, G=0.0, rc2=RC2, collide=True)
    assert counts.tolist() == [6] * 6 and alive.all()
    assert np.array_equal(st, init.astype(np.float32))


def test_mass_conserved_exactly_and_counts_monotone():
    kw = dict(G=2.0 ** -24, dt=0.25, eps2=2.0 ** -18, rc2=2.0 ** -12, collide=True)
    s0, _, _, _ = oracle.nbody_run(1500, 0, 9, **kw)
    s, alive, counts, _ = oracle.nbody_run(1500, 20, 9, **kw)
    assert float(s[alive == 1, 4].astype(np.float64).sum()) == float(s0[:, 4].astype(np.float64).sum())
    assert np.all(np.diff(counts.astype(np.int64)) <= 0) and counts[-1] < counts[0]
    assert counts[-1] == alive.sum()
    assert np.all(s[alive == 0] == 0)


@pytest.mark.parametrize("collide", [False, True])
def test_order_independence(collide):
    kw = dict(G=2.0 ** -22, dt=0.25, eps2=2.0 ** -18, rc2=2.0 ** -12, collide=collide)
    ref = oracle.nbody_run(700, 8, 3, **kw)
    for os_ in (1, 77, 12345):
        got = oracle.nbody_run(700, 8, 3, order_seed=os_, **kw)
        for a, b in zip(ref, got):
            assert np.array_equal(a, b)


def test_initial_draw():
    n, vs = 20000, 2.0 ** -8
    s, alive, counts, _ = oracle.nbody_run(n, 0, 0x5EED0006, G=0.0, dt=0.25, eps2=1.0, vscale=vs,
                                           mass_max=16)
    assert counts.tolist() == [n] and alive.all()
    assert s[:, :2].min() >= -1 and s[:, :2].max() < 1
    assert np.abs(s[:, 2:4]).max() <= vs / 2
    assert abs(s[:, 0].mean()) < 5 * (1 / math.sqrt(3)) / math.sqrt(n)
    m = s[:, 4]
    assert np.array_equal(m, np.round(m)) and m.min() == 1 and m.max() == 16
    hist = np.bincount(m.astype(int), minlength=17)[1:]
    assert np.all(np.abs(hist - n / 16) < 5 * math.sqrt(n / 16))
    # distinct draws per body: no two bodies share a position
    assert len({(a, b) for a, b in s[:, :2].tolist()}) == n


def test_force_on_single_bodies():
    # closed form of the pair at rest, on the fixed-point grid
    G, a, m, eps2 = 2.0 ** -10, 0.25, 2.0, 2.0 ** -6
    st = np.array([[-a, 0, 0, 0, m], [a, 0, 0, 0, m]], np.float32)
    f = oracle.nbody_force_on(st, [0, 1], G=G, eps2=eps2)
    d2 = (2 * a) ** 2 + eps2
    assert f[0, 0] == pytest.approx(G * m * m * 2 * a / d2 ** 1.5 * S, rel=1e-6)
    assert f[1, 0] == -f[0, 0] and f[0, 1] == 0 and f[1, 1] == 0
    # the forces of a random state sum to zero, and the first step of a run moves
    # each body by exactly those forces
    kw = dict(G=2.0 ** -20, eps2=2.0 ** -18)
    s0, _, _, _ = oracle.nbody_run(300, 0, 21, dt=0.25, **kw)
    F = oracle.nbody_force_on(s0, range(300), **kw)
    assert np.all(F.sum(0) == 0) and np.abs(F).max() > 0
    s1, _, _, _ = oracle.nbody_run(300, 1, 21, dt=0.25, **kw)
    f32 = np.float32
    ax = (F[:, 0].astype(f32) * f32(2.0 ** -40)) / s0[:, 4]
    vx = s0[:, 2] + ax * f32(0.25)
    assert np.array_equal(s1[:, 2], vx)
    # dead bodies exert no force
    alive = np.ones(300, np.uint8)
    alive[::2] = 0
    Fa = oracle.nbody_force_on(s0, [1], alive, **kw)
    assert Fa[0, 0] == oracle.nbody_force_on(s0[1::2], [0], **kw)[0, 0]
