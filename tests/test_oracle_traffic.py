"""Pins of the oracle's batched Nagel-Schreckenberg rings.

Nagel & Schreckenberg (J. Phys. I France 2, 1992): with slow-down probability 0 the
model is deterministic; a lone car accelerates by one cell per step up to vmax = 5,
and the steady flow on a ring of density rho is J = min(rho * vmax, 1 - rho).
"""
import numpy as np

import oracle


def ring(L, cars, v=None):
    occ = np.zeros(L, np.uint8)
    occ[list(cars)] = 1
    vel = np.zeros(L, np.uint8)
    if v is not None:
        vel[list(cars)] = v
    return occ, vel


def test_lone_car_accelerates_to_vmax():
    L = 200
    occ, vel = ring(L, [10])
    pos = 10
    for t in range(1, 12):
        o, v, cars = oracle.traffic_run([L], [0], t, slow_thr=0, ramp_thr=0,
                                        init_occ=occ, init_v=vel)
        pos += min(t, 5)
        assert np.nonzero(o)[0].tolist() == [pos % L]
        assert v[pos % L] == min(t, 5)
        assert np.all(cars == 1)


def _mean_speed(L, rho, steps, seed):
    rng = np.random.default_rng(seed)
    n = int(rho * L)
    pos = np.sort(rng.choice(L, n, replace=False))
    occ, vel = ring(L, pos)
    o, v, _ = oracle.traffic_run([L], [0], steps, slow_thr=0, ramp_thr=0,
                                 init_occ=occ, init_v=vel)
    assert o.sum() == n
    return v[o.astype(bool)].mean()


def test_deterministic_free_flow_branch():
    # rho < 1/(vmax+1): every car ends at vmax
    assert _mean_speed(600, 0.10, 800, 1) == 5.0


def test_deterministic_congested_branch():
    # rho > 1/(vmax+1): J = 1 - rho, i.e. mean speed (1 - rho) / rho
    rho = 0.5
    assert abs(_mean_speed(600, rho, 1500, 2) - (1 - rho) / rho) < 1e-9
    rho = 0.25
    assert abs(_mean_speed(800, rho, 3000, 3) - (1 - rho) / rho) < 1e-9


def test_no_ramps_conserves_cars():
    L = [64, 100, 37]
    thr = [int(0.3 * 2**32)] * 3
    _, _, cars = oracle.traffic_run(L, thr, 50, seed=5, ramp_thr=0)
    assert np.all(cars == cars[0])


def brute_force(L, thr, steps, seed, slow_thr, ramp_thr):
    """Direct array simulation of the same rules, one ring at a time."""
    key = [seed & 0xFFFFFFFF, seed >> 32]
    w0 = lambda c: int(oracle.philox4x32(c, key)[0])
    occ_all, v_all, counts = [], [], []
    for i, Li in enumerate(L):
        occ = np.array([w0([0xFFFFFFFF, j, i, 0]) < thr[i] for j in range(Li)], np.uint8)
        v = np.zeros(Li, np.int64)
        cnt = [int(occ.sum())]
        for t in range(steps):
            nocc = np.zeros(Li, np.uint8)
            nv = np.zeros(Li, np.int64)
            for j in np.nonzero(occ)[0]:
                s = min(v[j] + 1, 5)
                d = 1
                while d <= s and not occ[(j + d) % Li]:
                    d += 1
                s = min(s, d - 1)
                if s > 0 and w0([t, j, i, 1]) < slow_thr:
                    s -= 1
                np_ = (j + s) % Li
                if np_ == Li // 2 and w0([t, Li // 2, i, 2]) < ramp_thr:
                    continue
                nocc[np_] = 1
                nv[np_] = s
            if nocc[0] == 0 and w0([t, 0, i, 3]) < ramp_thr:
                nocc[0] = 1
                nv[0] = 0
            occ, v = nocc, nv
            cnt.append(int(occ.sum()))
        occ_all.append(occ)
        v_all.append(v)
        counts.append(cnt)
    return np.concatenate(occ_all), np.concatenate(v_all), np.array(counts).T


def test_brute_force_small_rings():
    L = [16, 16, 23]
    thr = [int(0.3 * 2**32), int(0.6 * 2**32), int(0.2 * 2**32)]
    seed = 0x5EED0004
    # exaggerated ramp rate so that ramp events happen on such small rings
    o, v, cars = oracle.traffic_run(L, thr, 30, seed=seed, ramp_thr=int(0.5 * 2**32))
    bo, bv, bc = brute_force(L, thr, 30, seed, oracle.SLOW_THR, int(0.5 * 2**32))
    assert np.array_equal(o, bo)
    assert np.array_equal(v, bv.astype(np.uint8))
    assert np.array_equal(cars, bc)


def test_order_independence():
    L = [300, 513, 4096]
    thr = [int(0.1 * 2**32), int(0.2 * 2**32), int(0.3 * 2**32)]
    a = oracle.traffic_run(L, thr, 40, seed=3)
    b = oracle.traffic_run(L, thr, 40, seed=3, order_seed=17)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_rings_are_independent_of_the_batch():
    # replaying ring k of a batch alone (first_ring = k) reproduces its state
    L = [300, 513, 1000]
    thr = [int(0.1 * 2**32), int(0.2 * 2**32), int(0.3 * 2**32)]
    o, v, cars = oracle.traffic_run(L, thr, 60, seed=8)
    base = np.concatenate([[0], np.cumsum(L)])
    for k in range(3):
        ok, vk, ck = oracle.traffic_run([L[k]], [thr[k]], 60, seed=8, first_ring=k)
        assert np.array_equal(ok, o[base[k]:base[k + 1]])
        assert np.array_equal(vk, v[base[k]:base[k + 1]])
        assert np.array_equal(ck[:, 0], cars[:, k])
