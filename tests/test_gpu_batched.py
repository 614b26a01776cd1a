"""Persistent batched correlation: bitwise equal to plain launches, oracle
parity on the 256-image workload, per-bucket tuning (GPU)."""
import numpy as np
import pytest

from gpu_helpers import MAX_REL, max_rel_err, oracle_ref
from paper_2211_07260_gb300 import api, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def device_entries(probs, guard=-7.0, pitch_align=4):
    ents, outs = [], []
    for p in probs:
        d_in = torch.from_numpy(p.inp).cuda()
        pitch = (p.out_w + pitch_align - 1) // pitch_align * pitch_align
        out = torch.full((p.out_h, pitch), guard, dtype=torch.float32, device="cuda")
        ents.append((d_in, p.filt, out, p.out_h, p.out_w))
        outs.append(out)
    return ents, outs


def mixed_problems(n=40, seed=5):
    probs = synth.batch_problems(n, seed, lo=17, hi=300)
    # a non-multiple-of-4 pitch (scalar path) and a 1x1 filter
    probs.append(synth.conv_problem(33, 45, 9, seed=[seed, 99], pitch_align=1))
    probs.append(synth.conv_problem(70, 64, 1, seed=[seed, 98]))
    return probs


@pytest.mark.parametrize("mode", ["persistent", "launches"])
@pytest.mark.parametrize("tiles", [None, "varied", "tall"])
def test_batched_equals_plain_bitwise_and_oracle(tiles, mode):
    probs = mixed_problems()
    t = None
    if tiles == "varied":
        t = {}
        for i, k in enumerate(range(1, 18, 2)):
            t[(0, k)] = ((16, 32, 64, 128)[i % 4], (1, 2, 4)[i % 3])
            t[(1, k)] = ((128, 64, 32, 16)[i % 4], (4, 1, 2)[i % 3])
        # launches graph: per-bucket single-image blocks and tile heights
        for i, k in enumerate(range(1, 18, 2)):
            t[("L0", k)] = ((16, 32, 64, 128)[i % 4], (8, 4, 2, 1)[i % 4], (4, 2, 1)[i % 3])
    elif tiles == "tall":
        # 8-row tiles (filter sides <= 3 only; larger sides fall back to the
        # default tile)
        t = {(c, k): (32 if k < 5 else 64, 8) for c in (0, 1) for k in range(1, 18, 2)}
    ents, outs = device_entries(probs)
    ents_p, outs_p = device_entries(probs)
    with api.Batch(ents, t, mode=mode) as b, api.Batch(ents_p, t, mode="persistent") as bp:
        st = b.info()
        assert st["mode_name"] == mode and st["has_launch_graph"] == (mode == "launches")
        # one persistent kernel per filter-side class, each grid capped by its items
        assert st["n_images"] == len(probs) and st["n_items"] >= st["grid"] > 0
        classes = {0 if p.filt.shape[0] <= 7 else 1 if p.filt.shape[0] <= 11 else 2 for p in probs}
        assert st["launches"] == len(classes)
        b.run()
        bp.run_plain()
        torch.cuda.synchronize()
        for p, o, op in zip(probs, outs, outs_p):
            a = o.cpu().numpy()
            c = op.cpu().numpy()
            assert np.all(a[:, p.out_w:] == -7.0)            # pitch guard untouched
            assert np.array_equal(a[:, :p.out_w], c[:, :p.out_w])
            assert max_rel_err(a[:, :p.out_w], oracle_ref(p)) <= MAX_REL
        # a second replay gives the same bits
        b.run()
        torch.cuda.synchronize()
        for p, o, op in zip(probs, outs, outs_p):
            assert np.array_equal(o.cpu().numpy()[:, :p.out_w], op.cpu().numpy()[:, :p.out_w])
    assert api.status_read(clear=True) == 0


def test_empty_images_and_errors():
    p = synth.conv_problem(20, 20, 5, seed=1)
    d_in = torch.from_numpy(p.inp).cuda()
    out = torch.zeros((20, 20), dtype=torch.float32, device="cuda")
    with api.Batch([(d_in, p.filt, out, 0, 20), (d_in, p.filt, out, 20, 20)]) as b:
        assert b.info()["n_images"] == 1
        b.run()
    torch.cuda.synchronize()
    assert max_rel_err(out.cpu().numpy(), oracle_ref(p)) <= MAX_REL
    with pytest.raises(api.ConvTuneError):
        api.Batch([(d_in, np.ones((4, 4), np.float32), out, 20, 20)])  # even side
    with api.Batch([]) as b:
        b.run()


def test_workload_256_images_oracle_parity():
    probs = synth.batch_problems(256, seed=2)
    ents, outs = device_entries(probs)
    ents_q, outs_q = device_entries(probs)
    with api.Batch(ents) as b, api.Batch(ents_q) as bq:
        st = b.info()
        # images of this workload average ~0.7 M outputs: the automatic mode
        # replays the launches graph
        assert st["mode_name"] == "launches" and st["has_launch_graph"] == 1
        b.run()
        bq.run(which="persistent")
        torch.cuda.synchronize()
    flop = sum(2 * p.fh * p.fw * p.out_h * p.out_w for p in probs)
    assert st["flop"] == pytest.approx(flop)
    worst = 0.0
    for p, o, oq in zip(probs, outs, outs_q):
        a = o.cpu().numpy()[:, :p.out_w]
        assert np.array_equal(a, oq.cpu().numpy()[:, :p.out_w])  # both graphs, same bits
        worst = max(worst, max_rel_err(a, oracle_ref(p)))
    assert worst <= MAX_REL
    assert api.status_read(clear=True) == 0


def test_bucket_tuning_and_measurement():
    probs = synth.batch_problems(24, seed=7, lo=64, hi=700)
    ents, outs = device_entries(probs)
    tiles, recs = api.batch_tune(ents, "energy", api.measure_options(window_s=0.2, warmup_s=0.05))
    ks = {(int(p.out_h * p.out_w >= 512 * 512), p.fh) for p in probs}
    assert set(tiles) == ks
    # 4 block widths x tile heights 1, 2, 4 (and 8 for filter sides <= 3)
    assert len(recs) == sum(16 if k <= 3 else 12 for _, k in ks)
    for (cls, k), (bx, ty) in tiles.items():
        assert bx in (16, 32, 64, 128) and ty in ((1, 2, 4, 8) if k <= 3 else (1, 2, 4))
    with api.Batch(ents, tiles) as b:
        o = api.measure_options(window_s=0.2, warmup_s=0.05)
        recs_m = {w: b.measure(w, o) for w in ("default", "plain", "persistent", "launches")}
        for r in recs_m.values():
            assert r["gflops"] > 0 and r["energy_j"] > 0
    with api.Batch(ents, tiles, mode="persistent") as b:
        assert b.info()["has_launch_graph"] == 0
        with pytest.raises(api.ConvTuneError):
            b.measure("launches", o)
    torch.cuda.synchronize()
    for p, o in zip(probs, outs):
        assert max_rel_err(o.cpu().numpy()[:, :p.out_w], oracle_ref(p)) <= MAX_REL


def test_launches_tuning():
    probs = synth.batch_problems(20, seed=9, lo=64, hi=700)
    probs.append(synth.conv_problem(90, 77, 5, seed=[9, 99], pitch_align=1))  # no TMA
    ents, outs = device_entries(probs)
    start = {(0, 5): (64, 2), ("claim", 0): 2}
    tiles, recs = api.batch_tune_launches(ents, "energy",
                                          api.measure_options(window_s=0.1, warmup_s=0.05),
                                          start=start)
    ks = {(int(p.out_h * p.out_w >= 512 * 512), p.fh) for p in probs}
    assert {key for key in tiles if key[0] in ("L0", "L1")} == {(f"L{c}", k) for c, k in ks}
    assert tiles[(0, 5)] == (64, 2) and tiles[("claim", 0)] == 2  # other entries kept
    assert len(recs) == 9 * len(ks)
    for key, val in tiles.items():
        if key[0] in ("L0", "L1"):
            assert tuple(val) in {(16, 8, 4), (32, 4, 4), (32, 2, 4), (16, 4, 4), (64, 2, 4),
                                    (32, 8, 2), (32, 4, 2), (64, 4, 2), (128, 2, 2)}
    ents_p, outs_p = device_entries(probs)
    with api.Batch(ents, tiles, mode="launches") as b, api.Batch(ents_p, tiles) as bp:
        b.run()
        bp.run_plain()
        torch.cuda.synchronize()
    for p, o, op in zip(probs, outs, outs_p):
        a = o.cpu().numpy()[:, :p.out_w]
        assert np.array_equal(a, op.cpu().numpy()[:, :p.out_w])
        assert max_rel_err(a, oracle_ref(p)) <= MAX_REL
    assert api.status_read(clear=True) == 0


def test_many_images_fill_every_parameter_block_then_fall_back():
    # 6000 one-output 17x17 images: their taps fill a parameter block every
    # 23 images, so the launches run out (254 per batch) and the last images
    # read their taps from shared memory; 8 graph branches carry the
    # launches.  Every output still equals the plain launch, bit for bit.
    n = 6000
    probs = [synth.conv_problem(1, 1, 17, seed=[11, i]) for i in range(n)]
    ents, outs = device_entries(probs)
    ents_p, outs_p = device_entries(probs)
    with api.Batch(ents, None) as b, api.Batch(ents_p, None) as bp:
        st = b.info()
        assert st["launches"] == 254
        # too many images for a launches graph: the persistent kernels run
        assert st["mode_name"] == "persistent" and st["has_launch_graph"] == 0
        b.run()
        bp.run_plain()
        torch.cuda.synchronize()
        got = torch.stack([o[:, :1] for o in outs]).cpu().numpy()
        ref = torch.stack([o[:, :1] for o in outs_p]).cpu().numpy()
    assert np.array_equal(got, ref)
    taps_sum = np.array([float((p.inp[:17, :17].astype(np.float64) * p.filt).sum()) for p in probs])
    assert np.max(np.abs(got.ravel() - taps_sum) / np.abs(taps_sum)) <= MAX_REL
    assert api.status_read(clear=True) == 0
