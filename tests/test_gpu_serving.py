"""Serving over a resident kernel: requests arriving as a Poisson process are
admitted to free stream slots within a memory budget while others run; each
request's result equals the oracle's and equals the same request served
alone. GPU only."""
import numpy as np
import pytest
import torch

import streamgen as sg
from oracle import execute

import fpcheck

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2401_12377_b300 import build
    build.build()
    from paper_2401_12377_b300 import harness, serving



def _oracle(cat, k):
    sp = cat.specs[k]
    if sp.kind == "rl":
        _, b, _ = execute.run_rlsim(sg.RLSim(sp.seed, sp.rl), emit=True)
        return {"pos": b["pos"], "vel": b["vel"]}
    st = sg.dnn_stream(sp.seed, batch=sp.dnn_batch, blocks=sp.dnn_blocks,
                       weight_sets=sg.DNN_SERVE_WEIGHT_SETS, shared=cat.shared_host)
    return {"h": execute.run_inorder(st.buffers, st.tasks)["h"]}


def _close(g, o, exact):
    for k in o:
        if exact:
            assert np.array_equal(g[k].view(np.uint8), o[k].view(np.uint8)), k
    if not exact:
        fpcheck.assert_per_element(g, o, "served request")


@pytest.fixture(scope="module")
def cat():
    return serving.Catalogue(sg.serving_catalogue(3, n_types=10, lo=60, hi=600))


def test_mix_equals_alone_and_oracle(cat):
    n = 80
    arrivals, kinds = sg.poisson_arrivals(3, n, 2000.0, len(cat.specs))
    with harness.Context(32, n_streams=6, resident=True, capacity=1 << 12) as ctx:
        srv = serving.Server(cat, ctx)
        mix = srv.run(arrivals, kinds, keep=set(range(n)))
        assert (mix["latency_s"] > 0).all() and mix["tasks"].min() > 0
        alone = {}
        for k in sorted(set(int(x) for x in kinds)):
            r = srv.run(np.zeros(1), np.array([k]), keep={0})
            alone[k] = r["results"][0]
        ctx.stop()
        assert ctx.stats()["launches"] == 1
    for i in range(n):
        k = int(kinds[i])
        _close(mix["results"][i], alone[k], exact=True)      # same bits alone and in the mix
    for k in alone:
        _close(alone[k], _oracle(cat, k), exact=cat.specs[k].kind == "rl")


def test_budget_limits_memory_in_use(cat):
    """A budget of two of the largest blocks: requests wait for memory, the
    bytes in use never exceed it, every request still completes."""
    n = 40
    arrivals, kinds = sg.poisson_arrivals(9, n, 5000.0, len(cat.specs))
    budget = 2 * max(e.nbytes for e in cat.entries)
    with harness.Context(16, n_streams=8, resident=True) as ctx:
        srv = serving.Server(cat, ctx, budget_bytes=budget)
        r = srv.run(arrivals, kinds)
    assert r["peak_bytes"] <= budget
    assert (r["latency_s"] > 0).all()
    assert r["queue_s"].max() > 0            # some requests waited for memory


def test_server_restarts_slot_positions_when_idle(cat):
    """Every slot starts 300 positions below harness.REBASE_AT; once a slot is
    past it and no request is in flight, the server ends the resident launch,
    restarts the slots' positions at 0 and starts it again. Every request still
    completes with the oracle's results."""
    n = 40
    arrivals, kinds = sg.poisson_arrivals(5, n, 200.0, len(cat.specs))
    with harness.Context(32, n_streams=4, resident=True, capacity=1 << 12) as ctx:
        ctx.stop()
        for s in range(4):
            ctx.rebase(s, harness.REBASE_AT - 300)
        ctx.start()
        srv = serving.Server(cat, ctx)
        r = srv.run(arrivals, kinds, keep=set(range(n)))
        assert srv.restarts >= 1
        assert max(ctx.tail(s) for s in range(4)) < harness.REBASE_AT
        ctx.stop()
    assert r["tasks"].min() > 0
    for i in range(n):
        k = int(kinds[i])
        _close(r["results"][i], _oracle(cat, k), exact=cat.specs[k].kind == "rl")
