"""Pins for the oracle's task bodies and in-order executor: closed forms with
exactly representable data, invariants, brute force and graph search. CPU only."""
import random
from fractions import Fraction

import networkx as nx
import numpy as np
import pytest

import streamgen as sg
from oracle import addresses, deps, execute

f32 = np.float32
R = sg.Ref


def _run(op, bufs, arrays, scalars=None, ncta=1):
    out = {k: v.copy() for k, v in bufs.items()}
    execute.run_task(out, sg.Task(0, op, ncta, arrays, scalars or {}))
    return out


# --- elementwise and DNN bodies: exact integer data ---------------------------

def test_axpy_scale_add_exact():
    x = np.arange(-8, 8, dtype=np.float32)
    y = np.arange(16, dtype=np.float32) * 3
    b = {"x": x, "y": y, "z": np.zeros(16, np.float32)}
    out = _run("axpy", b, {"x": R("x", 0, 16), "y": R("y", 0, 16)}, {"a": f32(2)})
    assert np.array_equal(out["y"], 2 * np.arange(-8, 8) + 3 * np.arange(16))
    out = _run("scale", b, {"x": R("x", 2, 4), "y": R("y", 10, 4)}, {"a": f32(0.5)})
    want = y.copy(); want[10:14] = np.arange(-6, -2) * 0.5
    assert np.array_equal(out["y"], want)
    out = _run("add", b, {"x": R("x", 0, 16), "y": R("y", 0, 16), "z": R("z", 0, 16)})
    assert np.array_equal(out["z"], np.arange(-8, 8) + 3 * np.arange(16))


def test_inplace_axpy_aliases_exactly():
    y = np.array([1, 2, 3], np.float32)
    out = _run("axpy", {"y": y}, {"x": R("y", 0, 3), "y": R("y", 0, 3)}, {"a": f32(3)})
    assert np.array_equal(out["y"], [4, 8, 12])


def test_gemv_integer_exact_and_correctly_rounded():
    rng = np.random.default_rng(0)
    m, k = 7, 33
    W = rng.integers(-5, 6, (m, k)).astype(np.float32)
    x = rng.integers(-5, 6, k).astype(np.float32)
    out = _run("gemv", {"W": W.reshape(-1), "x": x, "y": np.zeros(m, np.float32)},
               {"W": R("W", 0, m * k), "x": R("x", 0, k), "y": R("y", 0, m)}, {"m": m, "k": k})
    assert np.array_equal(out["y"], (W.astype(np.int64) @ x.astype(np.int64)).astype(np.float32))
    # random fp32 data: the result is within half an fp32 ulp of the exact rational dot product
    W = rng.uniform(-1, 1, (4, 256)).astype(np.float32)
    x = rng.uniform(-1, 1, 256).astype(np.float32)
    out = _run("gemv", {"W": W.reshape(-1), "x": x, "y": np.zeros(4, np.float32)},
               {"W": R("W", 0, 1024), "x": R("x", 0, 256), "y": R("y", 0, 4)}, {"m": 4, "k": 256})
    for i in range(4):
        exact = sum(Fraction(float(W[i, j])) * Fraction(float(x[j])) for j in range(256))
        ulp = np.spacing(np.abs(out["y"][i]))
        assert abs(Fraction(float(out["y"][i])) - exact) <= Fraction(float(ulp)) / 2


def test_bias_relu_and_resid():
    t = np.array([-2, -1, 0, 1, 2, -0.0], np.float32)
    b = np.array([1, 1, 0, -1, 1, 0], np.float32)
    out = _run("bias_relu", {"t": t, "b": b}, {"t": R("t", 0, 6), "b": R("b", 0, 6)})
    assert np.array_equal(out["t"], [0, 0, 0, 0, 3, 0])
    assert not np.signbit(out["t"]).any()                 # relu(-0) is +0
    h = np.array([1, 2, 3], np.float32)
    out = _run("resid", {"h": h, "u": np.array([4, 5, 6], np.float32), "b": np.array([1, 1, 1], np.float32)},
               {"h": R("h", 0, 3), "u": R("u", 0, 3), "b": R("b", 0, 3)})
    assert np.array_equal(out["h"], [6, 8, 10])


def test_sleep_body_update():
    out = _run("sleep", {"y": np.array([6, 9], np.float32)}, {"y": R("y", 0, 1)}, {"ns": 0, "tag": f32(2)})
    assert np.array_equal(out["y"], [5, 9])


# --- rigid-sphere bodies ------------------------------------------------------

S = sg.RL_SPHERES


def _env(pos, radius, invmass, vel=None):
    prop = np.stack([radius, invmass], -1).astype(np.float32)
    return {"pos": pos.astype(np.float32).reshape(-1), "prop": prop.reshape(-1),
            "vel": (np.zeros((S, 3)) if vel is None else vel).astype(np.float32).reshape(-1),
            "cont": np.zeros(sg.RL_REC_BYTES, np.uint8), "nisl": np.zeros(1, np.uint32)}


def _bp(b):
    return _run("rl_broadphase", b, {"pos": R("pos", 0, S * 3), "prop": R("prop", 0, S * 2),
                                     "cont": R("cont", 0, sg.RL_REC_BYTES), "nisl": R("nisl", 0, 1)},
                {"nenv": np.uint32(1)})


def _decode(cont):
    nc = int(cont[0:4].view(np.uint32)[0]); ni = int(cont[4:8].view(np.uint32)[0])
    label = cont[8:40].copy(); root = cont[40:72][:ni].copy()
    pair = cont[72:72 + 2 * 496].view(np.uint16)[:nc]
    return nc, ni, label, root, [(int(p) & 255, int(p) >> 8) for p in pair]


@pytest.mark.parametrize("seed", range(6))
def test_broadphase_vs_brute_force_and_components(seed):
    rng = np.random.default_rng(seed)
    radius = rng.uniform(0.05, 0.1, S)
    pos = rng.uniform(0.1, 0.8, (S, 3))
    out = _bp(_env(pos, radius, np.ones(S)))
    nc, ni, label, root, pairs = _decode(out["cont"])
    p32, r32 = pos.astype(np.float32).astype(np.float64), radius.astype(np.float32).astype(np.float64)
    want, unsure = [], 0
    for i in range(S):
        for j in range(i + 1, S):
            d2 = float(np.sum((p32[j] - p32[i]) ** 2)); rs2 = (r32[i] + r32[j]) ** 2
            if abs(d2 - rs2) < 1e-5 * rs2:
                unsure += 1
                continue
            if d2 < rs2:
                want.append((i, j))
    assert unsure == 0
    assert pairs == want                                  # lexicographic order
    g = nx.Graph(); g.add_nodes_from(range(S)); g.add_edges_from(pairs)
    comps = [c for c in nx.connected_components(g)]
    for c in comps:
        for v in c:
            assert label[v] == min(c)
    islands = sorted(min(c) for c in comps if len(c) > 1)
    assert ni == len(islands) and list(root) == islands and out["nisl"][0] == ni


def _pair_env(vi, vj, gap=-0.01, mi=1.0, mj=1.0):
    pos = np.tile([[5.0, 5.0, 5.0]], (S, 1)) + np.arange(S)[:, None] * 10.0  # far apart
    pos[0] = [1.0, 1.0, 1.0]
    pos[1] = [1.0 + 0.2 + gap, 1.0, 1.0]
    radius = np.full(S, 0.1)
    invm = np.ones(S); invm[0], invm[1] = mi, mj
    vel = np.zeros((S, 3)); vel[0], vel[1] = vi, vj
    return _env(pos, radius, invm, vel)


def _solve(b, beta_dt=f32(48.0), slop=f32(0.001)):
    b = _bp(b)
    return _run("rl_solve", b, {"pos": R("pos", 0, S * 3), "vel": R("vel", 0, S * 3),
                                "prop": R("prop", 0, S * 2), "cont": R("cont", 0, sg.RL_REC_BYTES)},
                {"beta_dt": beta_dt, "slop": slop})


def test_solve_symmetric_head_on_pair():
    b = _solve(_pair_env([1, 0, 0], [-1, 0, 0], gap=-0.001))
    v = b["vel"].reshape(S, 3)
    assert v[0, 0] == -v[1, 0] and v[0, 0] <= 0          # symmetric, separating
    assert np.all(v[:, 1:] == 0) and np.all(v[2:] == 0)   # only the normal component changes
    # with pen == slop the bias vanishes: the approach speed is removed exactly once
    assert abs(v[0, 0]) < 1e-6


def test_solve_conserves_momentum_of_an_island():
    rng = np.random.default_rng(3)
    pos = rng.uniform(0.2, 0.5, (S, 3))
    radius = rng.uniform(0.05, 0.1, S); invm = rng.uniform(0.5, 2.0, S)
    vel = rng.uniform(-1, 1, (S, 3))
    b0 = _env(pos, radius, invm, vel)
    b1 = _solve(b0)
    m = (1.0 / invm.astype(np.float32)).astype(np.float64)[:, None]
    p0 = (m * b0["vel"].reshape(S, 3)).sum(0); p1 = (m * b1["vel"].reshape(S, 3)).sum(0)
    assert np.allclose(p0, p1, rtol=0, atol=1e-4)
    assert not np.array_equal(b0["vel"], b1["vel"])        # contacts existed


@pytest.mark.parametrize("wi,wj", [(1.0, 1.0), (0.5, 2.0)])
def test_solve_resting_overlap_gets_the_bias_velocity_in_closed_form(wi, wj):
    """A resting pair that overlaps by more than the slop. The first sweep
    finds v_n = 0 and applies dl = beta_dt * (pen - slop) / (w_i + w_j); every
    later sweep then sees v_n equal to the bias and applies nothing. So the
    result, for any number of sweeps, is v_i = -dl * w_i * n, v_j = +dl * w_j * n
    and a relative normal velocity of exactly the Baumgarte bias: this pins the
    bias term's sign, factor and the slop's place in it."""
    beta_dt, slop = f32(48.0), f32(0.001)
    b = _solve(_pair_env([0, 0, 0], [0, 0, 0], gap=-0.01, mi=wi, mj=wj), beta_dt=beta_dt, slop=slop)
    v = b["vel"].reshape(S, 3).astype(np.float64)
    p = b["pos"].reshape(S, 3).astype(np.float64)
    dist = p[1, 0] - p[0, 0]
    pen = 0.2 - dist                                       # radii 0.1 + 0.1
    assert pen > float(slop)
    bias = float(beta_dt) * (pen - float(slop))
    dl = bias / (wi + wj)
    assert v[0, 0] == pytest.approx(-dl * wi, rel=1e-5)
    assert v[1, 0] == pytest.approx(dl * wj, rel=1e-5)
    assert v[1, 0] - v[0, 0] == pytest.approx(bias, rel=1e-5)
    assert np.all(v[:, 1:] == 0) and np.all(v[2:] == 0)
    # a pair overlapping by less than the slop gets no bias at all
    b = _solve(_pair_env([0, 0, 0], [0, 0, 0], gap=-0.0005), beta_dt=beta_dt, slop=slop)
    assert np.all(b["vel"] == 0)


def test_solve_chain_pins_eight_sequential_sweeps():
    """Three equal spheres in a row touching (contacts (0,1) then (1,2)), no
    bias (beta_dt = 0), sphere 0 moving at 1 toward the others. One
    Gauss-Seidel sweep maps (a, b, b) to ((a + b) / 2, (a + 3b) / 4,
    (a + 3b) / 4), so a - b shrinks by 4 per sweep while a + 2b = 1 (momentum):
    after s sweeps v0 = (1 + 2 * 4^-s) / 3 and v1 = v2 = (1 - 4^-s) / 3. Every
    value is a dyadic rational with at most 17 bits (normals are exactly
    (1, 0, 0)), so fp32 gives them exactly and only s = 8 matches; a Jacobi
    sweep, a reordered contact list or another sweep count all give other
    values."""
    pos = np.tile([[5.0, 5.0, 5.0]], (S, 1)) + np.arange(S)[:, None] * 10.0
    pos[0] = [1.0, 1.0, 1.0]
    pos[1] = [1.1875, 1.0, 1.0]
    pos[2] = [1.375, 1.0, 1.0]
    radius = np.full(S, 0.125)
    vel = np.zeros((S, 3)); vel[0, 0] = 1.0
    b = _bp(_env(pos, radius, np.ones(S), vel))
    nc, ni, _, _, pairs = _decode(b["cont"])
    assert pairs == [(0, 1), (1, 2)] and ni == 1
    out = _solve(_env(pos, radius, np.ones(S), vel), beta_dt=f32(0.0))
    v = out["vel"].reshape(S, 3)
    s = 8
    a = Fraction(1 + 2 * Fraction(1, 4 ** s), 3)
    bb = Fraction(1 - Fraction(1, 4 ** s), 3)
    assert a.denominator <= 2 ** 17 and bb.denominator <= 2 ** 17
    assert Fraction(float(v[0, 0])) == a
    assert Fraction(float(v[1, 0])) == bb and Fraction(float(v[2, 0])) == bb
    for other in (7, 9):      # neighbouring sweep counts give different exact values
        assert Fraction(1 + 2 * Fraction(1, 4 ** other), 3) != a
    assert np.all(v[:, 1:] == 0) and np.all(v[3:] == 0)


def test_solve_without_contacts_is_identity():
    b = _pair_env([1, 0, 0], [-1, 0, 0], gap=0.5)
    out = _solve(b)
    assert np.array_equal(out["vel"], b["vel"])


def _integrate(b, steps, dt=f32(1 / 240), g=f32(-9.81), box=f32(10.0)):
    gdt = f32(g * dt)
    for _ in range(steps):
        b = _run("rl_integrate", b, {"pos": R("pos", 0, S * 3), "vel": R("vel", 0, S * 3),
                                     "prop": R("prop", 0, S * 2)},
                 {"nenv": np.uint32(1), "dt": dt, "gdt": gdt, "box": box})
    return b


def test_integrate_free_fall_closed_form():
    pos = np.full((S, 3), 5.0); radius = np.full(S, 0.1)
    b = _integrate(_env(pos, radius, np.ones(S)), 24)
    dt, gdt = 1 / 240, np.float32(np.float32(-9.81) * np.float32(1 / 240))
    n = 24
    vz = b["vel"].reshape(S, 3)[:, 2]; pz = b["pos"].reshape(S, 3)[:, 2]
    assert np.allclose(vz, n * float(gdt), rtol=1e-5)
    assert np.allclose(pz, 5.0 + dt * float(gdt) * n * (n + 1) / 2, rtol=1e-6)
    assert np.all(b["pos"].reshape(S, 3)[:, :2] == 5.0)


def test_integrate_floor_clamps_and_reflects():
    pos = np.full((S, 3), 5.0); pos[:, 2] = 0.1005
    radius = np.full(S, 0.1)
    vel = np.zeros((S, 3)); vel[:, 2] = -2.0
    b = _integrate(_env(pos, radius, np.ones(S), vel), 1)
    assert np.all(b["pos"].reshape(S, 3)[:, 2] == np.float32(0.1))
    vz_before = np.float32(np.float32(-2.0) + np.float32(np.float32(-9.81) * np.float32(1 / 240)))
    assert np.all(b["vel"].reshape(S, 3)[:, 2] == vz_before * np.float32(-0.5))


# --- stream executor: schedule independence over E ---------------------------

def _random_topo(n, E, rng):
    preds = {j: set() for j in range(n)}
    for i, j in E:
        preds[j].add(i)
    done, order = set(), []
    while len(order) < n:
        ready = [j for j in range(n) if j not in done and preds[j] <= done]
        j = rng.choice(ready)
        order.append(j); done.add(j)
    return order


@pytest.mark.parametrize("kind", ["elementwise", "ranges", "dnn"])
def test_any_topological_order_of_E_reproduces_in_order(kind):
    s = {"elementwise": lambda: sg.elementwise_stream(11),
         "ranges": lambda: sg.elementwise_stream(12, ranges=True),
         "dnn": lambda: sg.dnn_stream(13, batch=4, blocks=6)}[kind]()
    E = deps.full_dag(addresses.stream_segments(s.tasks, s.buffers))
    ref = execute.run_inorder(s.buffers, s.tasks)
    rng = random.Random(1)
    for _ in range(5):
        out = execute.run_inorder(s.buffers, s.tasks, _random_topo(len(s.tasks), E, rng))
        for k in ref:
            assert np.array_equal(ref[k], out[k])


def test_planted_mistake_literal_alg1_breaks_schedule_independence():
    """Plant the mistake on the CPU: drop RAW (Alg. 1 read literally). Some
    order allowed by that DAG must then change the result."""
    s = sg.elementwise_stream(21)
    segs = addresses.stream_segments(s.tasks, s.buffers)
    E_lit = set()
    for j in range(len(segs)):
        for i in range(j):
            if any(deps.overlap(a, b) for a in segs[j][1] for b in segs[i][0] + segs[i][1]):
                E_lit.add((i, j))
    ref = execute.run_inorder(s.buffers, s.tasks)
    rng = random.Random(2)
    differs = False
    for _ in range(20):
        out = execute.run_inorder(s.buffers, s.tasks, _random_topo(len(s.tasks), E_lit, rng))
        differs |= any(not np.array_equal(ref[k], out[k]) for k in ref)
    assert differs


def test_rl_stream_is_input_dependent_and_deterministic():
    p = sg.RLParams(n_env=16, steps=4, chunk=8)
    t1, b1, s1 = execute.run_rlsim(sg.RLSim(5, p))
    t2, b2, s2 = execute.run_rlsim(sg.RLSim(5, p))
    assert s1 == s2 and all(np.array_equal(b1[k], b2[k]) for k in b1)
    t3, _, _ = execute.run_rlsim(sg.RLSim(6, p))
    shape = lambda ts: [(t.op, t.ncta, tuple(sorted(t.arrays.items()))) for t in ts]
    assert shape(t1) == shape(t2)
    assert shape(t1) != shape(t3)                       # another seed, another task graph
