"""The step planner (kdt_config.plan) and the learned part in its batched form.

The planner only decides which warp takes which partition when (longest estimated work
first) and, with the learned proposal, evaluates the network for all moves before the
moves start; the triangulation must stay bit-exact with the oracle after every step, for
one instance and for a batch.  The learned form's hit rate and its gain over the same
steps without it are measured and printed (the benchmark reports them at full size)."""
import numpy as np
import pytest

from paper_2308_06484_gb300 import workloads as W
from tests.gpu_helpers import assert_same, run_kinetic
from tests.test_gpu_batch import _batch, _check_all, _step_moves

pytestmark = pytest.mark.gpu


def _tri(w, **kw):
    from paper_2308_06484_gb300 import kdt
    t = kdt.Triangulation(kdt.default_config(grid=w.grid, domain_bits=w.bits, **kw))
    t.build(w.positions)
    return t


@pytest.mark.parametrize("make", [
    lambda: W.c2(n=60000, grid=32, seed=51),
    lambda: W.KineticWorkload(W.mixture_lattice_points(60000, 24, 52), 16, 24, (1, 16), (1, 8), seed=53,
                              name="mixture"),
])
def test_planned_order_keeps_the_triangulation(make):
    w = make()
    t = _tri(w, plan=1)
    run_kinetic(t, w, 6, every=1)
    st = t.stats()
    assert st["fallbacks"] == 0 and st["moves"] > 0
    assert st["kernel_launches"] >= 5 * 6  # intake, planner (3), kinetic per step
    assert t.verify() == 0


def _trained(seed=61):
    """A proposal network trained briefly on its own traces (uniform points)."""
    import torch
    from paper_2308_06484_gb300 import kdt, proposal
    x, y = proposal.collect_traces([(W.c2(n=100000, grid=32, seed=seed), 25)], cap=200000)
    holder = kdt.Triangulation(kdt.default_config())
    tn = proposal.Trainer(holder, seed=0)
    tn.fit(x, y, epochs=4, batch=2048, seed=0)
    torch.cuda.synchronize()
    return tn, holder, y


def _steps_ms(t, moves, warmup=2):
    import torch
    for mv in moves[:warmup]:
        t.step(mv)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for mv in moves[warmup:]:
        t.step(mv)
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def test_learned_form_parity_hit_rate_and_gain():
    import torch
    tn, holder, ytrain = _trained()
    counts = np.bincount(ytrain[:, 0].cpu().numpy(), minlength=17)
    majority = counts.max() / counts.sum()
    # the same steps plain, with the in-move proposal, and with the planner's proposal
    w = W.c2(n=200000, grid=32, seed=62)
    xy0 = w.positions
    moves = [torch.from_numpy(w.next_moves()).cuda() for _ in range(12)]
    final = w.positions
    res = {}
    for name, kw, prop in (("plain", {}, False), ("in_move", {}, True), ("planned", {"plan": 2}, True)):
        from paper_2308_06484_gb300 import kdt
        t = kdt.Triangulation(kdt.default_config(grid=32, domain_bits=24, **kw))
        t.build(xy0)
        if prop:
            t.set_proposal(tn.params)
        ms = _steps_ms(t, moves)
        st = t.stats()
        assert_same(t.export_triangles(), final, name)
        assert t.verify() == 0
        res[name] = (ms, st)
        t.close()
    hit_in = res["in_move"][1]["proposal_hits"] / max(1, res["in_move"][1]["proposal_moves"])
    hit_pl = res["planned"][1]["proposal_hits"] / max(1, res["planned"][1]["proposal_moves"])
    # the network learned something beyond the most frequent slot, and the planner's
    # guesses (made on the stars at the start of the step) hit about as often
    assert hit_in > majority + 0.05, (hit_in, majority)
    assert hit_pl > hit_in - 0.05, (hit_pl, hit_in)
    gain_in = res["plain"][0] / res["in_move"][0] - 1.0
    gain_pl = res["plain"][0] / res["planned"][0] - 1.0
    print("learned proposal: hit rate in-move %.3f planned %.3f (majority slot %.3f); gain in-move %+.3f "
          "planned %+.3f" % (hit_in, hit_pl, majority, gain_in, gain_pl))
    holder.close()


def test_batched_learned_form_matches_oracle():
    import torch
    from paper_2308_06484_gb300 import kdt
    tn, holder, _ = _trained(seed=63)
    ws = _batch(16, 500, 8000, seed=64)
    t = kdt.Triangulation(kdt.default_config(domain_bits=20, plan=2))
    t.build_batch([w.positions for w in ws])
    t.set_proposal(tn.params)
    for s in range(6):
        mv, offs = _step_moves(ws)
        t.step_batch(torch.from_numpy(mv).cuda(), offs)
        if s % 2 == 1:
            _check_all(t, ws, "planned batch step %d" % s)
    st = t.stats()
    assert st["proposal_moves"] > 0 and st["proposal_hits"] > 0
    assert st["fallbacks"] == 0
    assert t.verify() == 0
    holder.close()
