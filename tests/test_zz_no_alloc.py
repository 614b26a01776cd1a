"""The batched entry point that allocates nothing (ct_batch_run_noalloc).

It exists for callers that may not allocate device memory -- code that runs
inside a framework or pool owning all of the GPU's memory, or after start-up
where allocating is forbidden because it can stall the device or fail.  This
file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process
(its first call on the device does the one-time set-up).
"""
import ctypes

import numpy as np
import pytest

from gpu_helpers import MAX_REL, max_rel_err, oracle_ref
from paper_2211_07260_gb300 import api, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _device(probs):
    ents, outs = [], []
    for p in probs:
        d_in = torch.from_numpy(p.inp).cuda()
        out = torch.full((p.out_h, (p.out_w + 3) // 4 * 4), -7.0, dtype=torch.float32,
                         device="cuda")
        ents.append((d_in, p.filt, out, p.out_h, p.out_w))
        outs.append(out)
    return ents, outs


def _run_noalloc(ents, stream):
    items, keep = api.batch_items(ents)
    rc = api.lib().ct_batch_run_noalloc(items, len(ents), None,
                                        ctypes.c_void_p(stream.cuda_stream))
    return rc, keep


def _noalloc_status(stream, clear=True):
    bits = ctypes.c_uint(0xFFFFFFFF)
    rc = api.lib().ct_batch_noalloc_status(ctypes.byref(bits), int(clear),
                                           ctypes.c_void_p(stream.cuda_stream))
    assert rc == api.CT_OK, api.lib().ct_last_error()
    return bits.value


@pytest.mark.parametrize("seed", [11])
def test_noalloc_matches_the_allocating_entry_point_on_two_calls(seed):
    stream = torch.cuda.Stream()
    # two different batches through the same fixed scratch, back to back
    batches = [synth.batch_problems(48, seed, lo=17, hi=400),
               synth.batch_problems(30, seed + 1, lo=100, hi=700)
               + [synth.conv_problem(33, 45, 9, seed=[seed, 7], pitch_align=1)]]
    staged = [(probs,) + _device(probs) for probs in batches]
    torch.cuda.synchronize()
    results = []
    keeps = []
    for probs, ents, outs in staged:
        rc, keep = _run_noalloc(ents, stream)
        keeps.append(keep)
        assert rc == api.CT_OK, api.lib().ct_last_error()
        # the kernels raised no error bit in this call
        assert _noalloc_status(stream) == 0
        results.append((probs, outs))
    stream.synchronize()
    # once set up (and its kernels loaded), further calls take no device
    # memory: neither from torch's caching allocator nor from the device
    reserved = torch.cuda.memory_reserved()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        for probs, ents, outs in staged:
            rc, keep = _run_noalloc(ents, stream)
            keeps.append(keep)
            assert rc == api.CT_OK, api.lib().ct_last_error()
    assert _noalloc_status(stream) == 0
    stream.synchronize()
    assert torch.cuda.memory_reserved() == reserved
    assert torch.cuda.mem_get_info()[0] == free0
    for probs, outs in results:
        ents_ref, outs_ref = _device(probs)
        with api.Batch(ents_ref) as b:
            b.run()
            torch.cuda.synchronize()
        for p, o, r in zip(probs, outs, outs_ref):
            got = o.cpu().numpy()
            ref = r.cpu().numpy()
            assert np.all(got[:, p.out_w:] == -7.0)
            assert max_rel_err(got[:, :p.out_w], ref[:, :p.out_w]) <= MAX_REL
            assert np.array_equal(got[:, :p.out_w], ref[:, :p.out_w])
            assert max_rel_err(got[:, :p.out_w], oracle_ref(p)) <= MAX_REL


def test_noalloc_rejects_more_images_than_the_scratch_holds():
    p = synth.conv_problem(8, 8, 3, seed=0)
    ents, outs = _device([p])
    stream = torch.cuda.Stream()
    rc, _ = _run_noalloc(ents * 257, stream)
    assert rc == api.CT_EINVAL
    assert b"limit 256" in api.lib().ct_last_error()
    rc, _ = _run_noalloc(ents * 256, stream)  # the limit itself is accepted
    stream.synchronize()
    assert rc == api.CT_OK
    assert _noalloc_status(stream) == 0
    assert max_rel_err(outs[0].cpu().numpy()[:, :8], oracle_ref(p)) <= MAX_REL
