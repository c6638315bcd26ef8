"""The allocation-free path search against the regular path tracer.

risrt_find_paths_noalloc serves callers that may not allocate device memory while they run (code
executing where the CUDA allocator must not be touched, or hosts that hand the library a fixed
memory budget). It runs the same reflected-path search as risrt_trace_paths but on a scratch array
built into the library, so its answers must be identical to what trace_paths exports: the Tx-leg
sequences between the Tx and the RIS centre, and the Tx->receiver environment sequences. Two calls
in a row must agree too, since every call reuses (and must first clear) the same array.

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_2402_13034_gb300 import scenarios as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def traced_room():
    import torch
    from paper_2402_13034_gb300 import build as B
    from paper_2402_13034_gb300 import risrt as R
    B.build()
    w = S.room(grid=6)
    ctx = R.Context(0, torch.cuda.current_stream().cuda_stream)
    scene, ris, rx = R.upload_workload(ctx, w)
    ps = ctx.trace_paths(scene, ris, rx, w.freq_hz, w.max_order_tx, w.max_order_rx, R.flags_of(w))
    exp = ps.export()
    torch.cuda.synchronize()
    return w, ctx, scene, exp


def test_tx_leg_matches_trace_paths_twice(traced_room):
    w, ctx, scene, exp = traced_room
    ref = np.sort(exp["tx_seqs"])
    for _ in range(2):
        ids = ctx.find_paths_noalloc(scene, w.tx.pos, -1, w.ris.center, w.ris.host_face, w.max_order_tx)
        assert np.array_equal(ids, ref)


def test_environment_paths_match_trace_paths_twice(traced_room):
    w, ctx, scene, exp = traced_room
    checked = 0
    for i in range(0, w.n_rx, 5):
        ref = np.sort(exp["env"][i])
        for _ in range(2):
            ids = ctx.find_paths_noalloc(scene, w.tx.pos, -1, w.rx_xyz[i], -1, w.max_order_rx)
            assert np.array_equal(ids, ref), i
        checked += len(ref) > 0
    assert checked > 0


def test_rejects_scene_beyond_static_scratch():
    import torch
    from paper_2402_13034_gb300 import risrt as R
    w = S.office(n_boxes=200)        # ~1,200 faces: order 2 needs far more than the static array
    ctx = R.Context(0, torch.cuda.current_stream().cuda_stream)
    sc = w.scene
    scene = ctx.scene_upload(sc.verts, sc.tris, sc.face_id, sc.mat_id, sc.mats)
    with pytest.raises(R.RisrtError) as e:
        ctx.find_paths_noalloc(scene, w.tx.pos, -1, w.ris.center, w.ris.host_face, 2)
    assert e.value.code == 6 and "static scratch" in str(e.value)


def test_trace_after_noalloc_retries_with_wide_slab():
    """Kernel attributes are shared by every caller in the process: a path search without allocation,
    then a trace whose receivers each have more geometric candidates than its first slab holds (two
    stacks of parallel plates), which retries with a wider slab and sorts it with more shared memory.
    The path search still matches, and the trace's path sets match the oracle."""
    import torch
    from paper_2402_13034_gb300 import risrt as R
    from tests.helpers import oracle_parity, run_gpu
    w = S.plate_corridor()
    ctx = R.Context(0, torch.cuda.current_stream().cuda_stream)
    scene, ris, rx = R.upload_workload(ctx, w)
    ids = ctx.find_paths_noalloc(scene, w.tx.pos, -1, w.ris.center, w.ris.host_face, w.max_order_tx)
    g = run_gpu(w)
    assert g["paths"]["stats"].n_candidates > 512 * w.n_rx
    assert np.array_equal(ids, np.sort(g["paths"]["tx_seqs"]))
    oracle_parity(w, g)
