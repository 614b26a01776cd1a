"""Parity of the CUDA correlation kernels with the FP64 oracle (GPU)."""
import itertools

import numpy as np
import pytest

from gpu_helpers import MAX_REL, max_rel_err, normwise_err, oracle_ref, to_device
from paper_2211_07260_gb300 import api, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BX, BY, T, VW = (16, 32, 64, 128), (1, 2, 4, 8), (1, 2, 4), (1, 2, 4)
STAGES = (api.STAGE_DIRECT, api.STAGE_SMEM, api.STAGE_TMA)
FILTS = (api.FILTER_SHARED, api.FILTER_CONST)


def full_space():
    for bx, by, tx, ty, st, fm, vw in itertools.product(BX, BY, T, T, STAGES, FILTS, VW):
        yield api.Config(bx, by, tx, ty, st, fm, vw)


def run(prob, cfg, d_in, d_out):
    api.conv2d_run(d_in, prob.filt, d_out, prob.out_h, prob.out_w, cfg)


@pytest.mark.parametrize("k", [1, 3, 5, 7, 9, 11, 13, 15, 17])
def test_every_config_matches_oracle_and_each_other_bitwise(k):
    # ragged sizes: several tiles of the largest CTA tile plus a tail
    prob = synth.conv_problem(75, 139, k, seed=100 + k)
    ref = oracle_ref(prob)
    d_in, full, d_out = to_device(prob, out_pitch=144, guard_rows=2)
    first = None
    n_run = n_pruned = 0
    ok_cfgs, pruned = set(), {}
    for cfg in full_space():
        rc, why = api.conv2d_check(d_in, prob.filt, d_out, prob.out_h, prob.out_w, cfg)
        if rc == api.CT_ECONFIG:
            n_pruned += 1
            pruned[cfg.as_tuple()] = why
            continue
        ok_cfgs.add(cfg.as_tuple())
        assert rc == api.CT_OK, (cfg, why)
        full.fill_(-7.0)
        run(prob, cfg, d_in, d_out)
        torch.cuda.synchronize()
        got = full.cpu().numpy()
        out = got[2:2 + prob.out_h, :prob.out_w]
        # guard band untouched: rows above/below and the pitch columns
        assert np.all(got[:2] == -7.0) and np.all(got[2 + prob.out_h:] == -7.0), cfg
        assert np.all(got[2:2 + prob.out_h, prob.out_w:] == -7.0), cfg
        if first is None:
            first = out.copy()
            assert max_rel_err(out, ref) <= MAX_REL
        else:
            assert np.array_equal(out.view(np.uint32), first.view(np.uint32)), cfg
        n_run += 1
    assert api.status_read(clear=True) == 0
    # TMA points pruned although the same point with cp.async staging runs
    tma_only = {c: w for c, w in pruned.items()
                if c[4] == api.STAGE_TMA and c[:4] + (api.STAGE_SMEM,) + c[5:] in ok_cfgs}
    n_tma_only_pruned = len(tma_only)
    # wide TMA tiles are staged as several boxes: only blocks the registers or
    # shared memory cannot hold are pruned, never a TMA point whose direct or
    # cp.async twin runs
    assert n_run > 1000
    assert n_tma_only_pruned == 0, tma_only


@pytest.mark.parametrize("shape", [(1, 1), (1, 37), (29, 1), (2, 2), (17, 17), (64, 64),
                                   (33, 65), (130, 7)])
@pytest.mark.parametrize("k", [3, 17])
def test_small_and_degenerate_shapes(shape, k):
    h, w = shape
    prob = synth.conv_problem(h, w, k, seed=[h, w, k])
    ref = oracle_ref(prob)
    d_in, full, d_out = to_device(prob)
    for cfg in (api.Config(16, 1, 1, 1, api.STAGE_DIRECT, api.FILTER_CONST, 1),
                api.Config(32, 8, 4, 4, api.STAGE_SMEM, api.FILTER_SHARED, 4),
                api.Config(32, 4, 4, 2, api.STAGE_TMA, api.FILTER_CONST, 4),
                api.Config(128, 2, 2, 4, api.STAGE_DIRECT, api.FILTER_SHARED, 2)):
        full.fill_(-7.0)
        run(prob, cfg, d_in, d_out)
        out = full.cpu().numpy()[:, :w]
        assert max_rel_err(out, ref) <= MAX_REL, cfg


@pytest.mark.parametrize("fh,fw", [(3, 5), (1, 7), (4, 4), (2, 6), (21, 21), (31, 3)])
def test_generic_kernel_non_square_and_large_filters(fh, fw):
    prob = synth.conv_problem(47, 53, fh | 1, fw | 1, seed=[fh, fw])
    # even sides: use the raw padded array with an even filter
    filt = np.random.default_rng([fh, fw]).random((fh, fw), dtype=np.float32)
    prob = synth.ConvProblem(inp=prob.inp, in_w=prob.in_w, filt=filt,
                             out_h=prob.in_h - fh + 1, out_w=prob.in_w - fw + 1)
    ref = oracle_ref(prob)
    d_in, full, d_out = to_device(prob)
    # every block shape of the space (the generic kernel takes one output per
    # thread and its taps from shared memory whatever the rest says): all the
    # same bits, within the gate of the oracle
    first = None
    for bx, by in itertools.product(BX, BY):
        full.fill_(-7.0)
        run(prob, api.Config(bx, by, 1, 1, api.STAGE_DIRECT, api.FILTER_SHARED, 1), d_in, d_out)
        got = full.cpu().numpy()
        assert np.all(got[:, prob.out_w:] == -7.0)
        out = got[:, :prob.out_w]
        if first is None:
            first = out.copy()
            assert max_rel_err(out, ref) <= MAX_REL
        else:
            assert np.array_equal(out, first), (bx, by)


def test_signed_values_normwise():
    prob = synth.conv_problem(200, 300, 9, seed=9, values="signed")
    ref = oracle_ref(prob)
    d_in, full, d_out = to_device(prob)
    for cfg in (api.Config(), api.Config(64, 2, 2, 1, api.STAGE_DIRECT, api.FILTER_CONST, 2)):
        run(prob, cfg, d_in, d_out)
        assert normwise_err(full.cpu().numpy()[:, :prob.out_w], ref) <= MAX_REL


def test_empty_output_is_a_no_op():
    prob = synth.conv_problem(4, 4, 3, seed=0)
    d_in, full, d_out = to_device(prob)
    full.fill_(5.0)
    api.conv2d_run(d_in, prob.filt, d_out, 0, prob.out_w, api.Config())
    api.conv2d_run(d_in, prob.filt, d_out, prob.out_h, 0, api.Config())
    assert torch.all(full == 5.0)


def test_alignment_and_pitch_rules():
    prob = synth.conv_problem(40, 41, 5, seed=1, pitch_align=1)  # pitch 45: not a multiple of 4
    ref = oracle_ref(prob)
    d_in = torch.from_numpy(prob.inp).cuda()
    out = torch.zeros((prob.out_h, 41), dtype=torch.float32, device="cuda")
    rc, why = api.conv2d_check(d_in, prob.filt, out, prob.out_h, prob.out_w,
                               api.Config(vec_width=4))
    assert rc == api.CT_ECONFIG and "aligned" in why
    rc, _ = api.conv2d_check(d_in, prob.filt, out, prob.out_h, prob.out_w,
                             api.Config(staging=api.STAGE_TMA, vec_width=1))
    assert rc == api.CT_ECONFIG
    for st in (api.STAGE_DIRECT, api.STAGE_SMEM):
        out.zero_()
        api.conv2d_run(d_in, prob.filt, out, prob.out_h, prob.out_w,
                       api.Config(staging=st, vec_width=1))
        assert max_rel_err(out.cpu().numpy(), ref) <= MAX_REL
    # misaligned base pointer (one float in): scalar loads still work
    prob4 = synth.conv_problem(40, 40, 5, seed=2)
    ref4 = oracle_ref(prob4)
    big = torch.zeros(prob4.inp.size + 4, dtype=torch.float32, device="cuda")
    big[1:1 + prob4.inp.size] = torch.from_numpy(prob4.inp.ravel()).cuda()
    shifted = big[1:1 + prob4.inp.size].view(prob4.inp.shape)
    out2 = torch.zeros((40, 40), dtype=torch.float32, device="cuda")
    rc, _ = api.conv2d_check(shifted, prob4.filt, out2, 40, 40, api.Config(vec_width=2))
    assert rc == api.CT_ECONFIG
    api.conv2d_run(shifted, prob4.filt, out2, 40, 40,
                   api.Config(staging=api.STAGE_DIRECT, vec_width=1))
    assert max_rel_err(out2.cpu().numpy(), ref4) <= MAX_REL


def test_invalid_arguments():
    prob = synth.conv_problem(8, 8, 3, seed=0)
    d_in, full, d_out = to_device(prob)
    bad = [api.Config(block_x=48), api.Config(block_x=8), api.Config(block_x=128, block_y=16),
           api.Config(tile_x=3), api.Config(staging=3), api.Config(filter_mem=2),
           api.Config(vec_width=8)]
    for cfg in bad:
        rc, _ = api.conv2d_check(d_in, prob.filt, d_out, 8, 8, cfg)
        assert rc == api.CT_ECONFIG, cfg
    with pytest.raises(api.ConvTuneError) as e:
        api.conv2d_run(d_in, prob.filt, d_out, 8, 8, api.Config(), in_pitch=5)
    assert e.value.status == api.CT_EINVAL
    rc, _ = api.conv2d_check(d_in, np.ones((33, 1), np.float32), d_out, 8, 8, api.Config())
    assert rc == api.CT_EINVAL


def test_grid_limit_is_reported():
    # out_h / (block_y * tile_y) beyond 65535 CTAs in y is pruned, not launched
    prob_h = 70000
    d_in = torch.zeros((prob_h + 2, 8), dtype=torch.float32, device="cuda")
    d_out = torch.zeros((prob_h, 4), dtype=torch.float32, device="cuda")
    filt = np.ones((3, 3), np.float32)
    rc, why = api.conv2d_check(d_in, filt, d_out, prob_h, 4,
                               api.Config(16, 1, 1, 1, api.STAGE_DIRECT, api.FILTER_CONST, 1))
    assert rc == api.CT_ECONFIG and "grid" in why
    rc, _ = api.conv2d_check(d_in, filt, d_out, prob_h, 4,
                             api.Config(16, 2, 1, 1, api.STAGE_DIRECT, api.FILTER_CONST, 1))
    assert rc == api.CT_OK


@pytest.mark.parametrize("shape", [(300, 257, 7), (1100, 300, 9), (4100, 96, 17)])
def test_host_entry_point_matches_device_run(shape):
    # several row bands for the larger shapes (copies overlap the kernels)
    h, w, k = shape
    prob = synth.conv_problem(h, w, k, seed=3)
    cfg = api.Config(32, 4, 4, 2, api.STAGE_SMEM, api.FILTER_CONST, 4)
    d_in, full, d_out = to_device(prob)
    run(prob, cfg, d_in, d_out)
    dev = full.cpu().numpy()
    host_out = np.full((prob.out_h, dev.shape[1]), -1.0, np.float32)
    api.conv2d_run_host(prob.inp, prob.filt, host_out, prob.out_h, prob.out_w, cfg)
    assert np.array_equal(host_out[:, :prob.out_w], dev[:, :prob.out_w])
    # pinned buffers (asynchronous, overlapping copies) give the same bits
    pin_in = torch.from_numpy(prob.inp).pin_memory().numpy()
    pin_out = torch.full(host_out.shape, -1.0).pin_memory().numpy()
    api.conv2d_run_host(pin_in, prob.filt, pin_out, prob.out_h, prob.out_w, cfg)
    assert np.array_equal(pin_out, host_out)
    assert np.all(host_out[:, prob.out_w:] == -1.0)  # padding columns untouched
    assert max_rel_err(host_out[:, :prob.out_w], oracle_ref(prob)) <= MAX_REL


def test_host_entry_point_explicit_bands():
    # any split of the rows gives the same bits as one launch; bad splits are
    # rejected before any copy
    prob = synth.conv_problem(700, 128, 5, seed=4)
    cfg = api.Config(32, 4, 4, 2, api.STAGE_TMA, api.FILTER_CONST, 4)
    ref = np.empty((700, 128), np.float32)
    api.conv2d_run_host(prob.inp, prob.filt, ref, 700, 128, cfg, bands=[700])
    assert max_rel_err(ref, oracle_ref(prob)) <= MAX_REL
    for split in ([1, 2, 697], [350, 350], [64] * 10 + [60], [699, 1], [11] * 63 + [7]):
        out = np.full((700, 128), -1.0, np.float32)
        api.conv2d_run_host(prob.inp, prob.filt, out, 700, 128, cfg, bands=split)
        assert np.array_equal(out, ref), split
    out = np.full((700, 128), -1.0, np.float32)
    for bad in ([700, 0], [350, 349], [350, 351], [10] * 70, [-1, 701]):
        with pytest.raises(api.ConvTuneError) as e:
            api.conv2d_run_host(prob.inp, prob.filt, out, 700, 128, cfg, bands=bad)
        assert e.value.status == api.CT_EINVAL
    assert np.all(out == -1.0)


@pytest.mark.parametrize("pinned", [True, False])
def test_host_entry_point_repeated_calls(pinned):
    # repeated calls on the same buffers (the library's device buffers and
    # streams are reused): every call must read the caller's current input
    # and give the same bits as a device run
    h, w, k = 1200, 256, 9
    cfg = api.Config(32, 4, 4, 2, api.STAGE_TMA, api.FILTER_CONST, 4)
    base = synth.conv_problem(h, w, k, seed=21)
    inp = np.empty_like(base.inp)
    out = np.empty((h, w), np.float32)
    if pinned:
        inp = torch.from_numpy(inp).pin_memory().numpy()
        out = torch.from_numpy(out).pin_memory().numpy()
    for rep in range(4):
        prob = synth.conv_problem(h, w, k, seed=[21, rep])
        prob = synth.ConvProblem(inp=prob.inp, in_w=prob.in_w, filt=base.filt,
                                 out_h=prob.out_h, out_w=prob.out_w)
        inp[...] = prob.inp
        out.fill(-1.0)
        api.conv2d_run_host(inp, base.filt, out, h, w, cfg)
        d_in, full, d_out = to_device(prob)
        run(prob, cfg, d_in, d_out)
        assert np.array_equal(out, full.cpu().numpy()[:, :w]), rep
    assert max_rel_err(out, oracle_ref(prob)) <= MAX_REL


@pytest.mark.parametrize("pinned", [True, False])
def test_host_entry_point_asynchronous_calls(pinned):
    # back-to-back asynchronous calls, each with its own input and output
    # (the library alternates two device buffer sets); the third
    # call is larger, so its buffer set is reallocated while the second call
    # may still run.  Every output equals the synchronous entry point's.
    cfg = api.Config(32, 4, 4, 2, api.STAGE_TMA, api.FILTER_CONST, 4)
    shapes = [(1100, 300, 7), (900, 260, 7), (1500, 400, 7), (1100, 300, 7), (300, 200, 5)]
    probs = [synth.conv_problem(h, w, k, seed=[31, i]) for i, (h, w, k) in enumerate(shapes)]
    ins, outs = [], []
    for p in probs:
        a = np.ascontiguousarray(p.inp)
        o = np.full((p.out_h, p.out_w), -1.0, np.float32)
        if pinned:
            a = torch.from_numpy(a).pin_memory().numpy()
            o = torch.from_numpy(o).pin_memory().numpy()
        ins.append(a)
        outs.append(o)
    for p, a, o in zip(probs, ins, outs):
        api.conv2d_run_host_async(a, p.filt, o, p.out_h, p.out_w, cfg)
    api.host_wait()
    for p, o in zip(probs, outs):
        ref = np.empty((p.out_h, p.out_w), np.float32)
        api.conv2d_run_host(p.inp, p.filt, ref, p.out_h, p.out_w, cfg)
        assert np.array_equal(o, ref)
        assert max_rel_err(o, oracle_ref(p)) <= MAX_REL
    # a synchronous call after an asynchronous one runs after it, and
    # returns with both outputs on the host
    (p0, a0, o0), (p1, a1, o1) = zip(probs[:2], ins[:2], outs[:2])
    o0.fill(-1.0)
    o1.fill(-1.0)
    api.conv2d_run_host_async(a0, p0.filt, o0, p0.out_h, p0.out_w, cfg)
    api.conv2d_run_host(a1, p1.filt, o1, p1.out_h, p1.out_w, cfg)
    assert max_rel_err(o0, oracle_ref(p0)) <= MAX_REL
    assert max_rel_err(o1, oracle_ref(p1)) <= MAX_REL
    api.host_wait()
    assert api.status_read(clear=True) == 0


@pytest.mark.parametrize("which", ["1024x1024_k7", "4096x4096_k17"])
def test_full_size_workloads(which):
    # the tuned configurations the bench times (energy- and time-optimal),
    # then others of the space; all must give the same bits
    if which == "1024x1024_k7":
        prob = synth.conv_problem(1024, 1024, 7, seed=0)
        cfgs = [api.Config(128, 4, 4, 4, api.STAGE_SMEM, api.FILTER_CONST, 4),
                api.Config(32, 4, 4, 2, api.STAGE_SMEM, api.FILTER_CONST, 4),
                api.Config(64, 8, 4, 4, api.STAGE_SMEM, api.FILTER_CONST, 4),
                api.Config(32, 8, 4, 4, api.STAGE_SMEM, api.FILTER_CONST, 4),
                api.Config(32, 4, 4, 4, api.STAGE_SMEM, api.FILTER_CONST, 4),
                api.Config(64, 2, 2, 2, api.STAGE_DIRECT, api.FILTER_CONST, 2),
                api.Config(128, 4, 4, 4, api.STAGE_TMA, api.FILTER_CONST, 4)]
    else:
        prob = synth.conv_problem(4096, 4096, 17, seed=1)
        cfgs = [api.Config(128, 8, 4, 2, api.STAGE_TMA, api.FILTER_CONST, 4),
                api.Config(32, 4, 4, 4, api.STAGE_TMA, api.FILTER_CONST, 4),  # 96 registers
                api.Config(16, 8, 4, 4, api.STAGE_TMA, api.FILTER_CONST, 4),  # 96 registers
                api.Config(32, 1, 4, 4, api.STAGE_TMA, api.FILTER_CONST, 4),
                api.Config(32, 8, 4, 4, api.STAGE_SMEM, api.FILTER_CONST, 4),
                api.Config(64, 2, 4, 4, api.STAGE_TMA, api.FILTER_CONST, 4)]
    ref = oracle_ref(prob)
    d_in, full, d_out = to_device(prob)
    outs = []
    for cfg in cfgs:
        full.fill_(-7.0)
        run(prob, cfg, d_in, d_out)
        outs.append(full.cpu().numpy()[:, :prob.out_w])
    assert max_rel_err(outs[0], ref) <= MAX_REL
    for o, cfg in zip(outs[1:], cfgs[1:]):
        assert np.array_equal(outs[0], o), cfg
    assert api.status_read(clear=True) == 0
