"""Forward parity: CUDA path (through the C ABI) vs the FP64 oracle.

Tolerance: err_max = max|F_gpu - F_ref| / max|F_ref| <= 1e-4 in fp32
(the target bound for the fp32 forward); fp32 rounding over ~2N merges
gives ~1e-6 in practice.
"""
import numpy as np
import pytest

import oracle
from paper_2505_02041_gb300 import scenes
from gpu_util import require_gpu, err_max, assert_fp32, to_dev, torch

pytestmark = pytest.mark.gpu

TOL = 1e-4


def _gpu_F(e, s, cascades=0, precision="fp32"):
    from paper_2505_02041_gb300 import HRC
    C, H, W = e.shape
    h = HRC(W, H, C, cascades, precision)
    F = h.forward(to_dev(e, torch.float32), to_dev(s, torch.float32))
    torch.cuda.synchronize()
    return h, F.cpu().numpy()


@pytest.mark.parametrize("W,H,C,casc,seed", [
    (64, 64, 1, 0, 0), (37, 23, 2, 0, 1), (5, 7, 1, 0, 2), (1, 6, 1, 0, 3), (1, 1, 1, 0, 4),
    (2, 2, 3, 0, 5), (128, 96, 3, 0, 6), (100, 100, 4, 0, 7), (64, 64, 1, 3, 8), (33, 65, 1, 0, 9),
    (257, 130, 1, 0, 10),
])
def test_forward_random_scenes(W, H, C, casc, seed):
    require_gpu()
    e, s = scenes.random_scene(W, H, C, seed)
    _, F = _gpu_F(e, s, casc)
    Fr = oracle.fluence(e, s, casc)
    assert_fp32(F, Fr)


def test_forward_disks64_scene():
    require_gpu()
    e, s = scenes.scene_by_name("disks64")
    _, F = _gpu_F(e, s)
    assert_fp32(F, oracle.fluence(e, s))


def test_forward_vacuum_is_zero():
    require_gpu()
    e = np.zeros((1, 40, 40), np.float32)
    s = np.zeros((40, 40), np.float32)
    s[10:20, 10:20] = 1e3
    _, F = _gpu_F(e, s)
    assert np.all(F == 0.0)


def t_live(n, x, k):
    """T_n(x, k) entries some fluence depends on: column 0 never (the sum reads
    R_0 at u + 1), T_0 only at odd columns (Eq. 14; even columns of level 0
    take T_1), T_1 at even columns only in even directions (Eqs. 15-17)."""
    if x == 0:
        return False
    if n == 0:
        return x % 2 == 1
    if n == 1:
        return x % 2 == 1 or k % 2 == 0
    return True


@pytest.mark.parametrize("q", range(4))
def test_levels_match_oracle(q):
    """Every T_n and R_n level of every quadrant frame, element by element.

    Entries no fluence depends on (column 0 of every level, the even columns
    of T_0, the odd directions of T_1 at even columns) are never computed and
    are exported as NaN; every other entry is compared."""
    require_gpu()
    e, s = scenes.random_scene(48, 40, 2, 12)
    h, _ = _gpu_F(e, s)
    U = 48 if q < 2 else 40
    N = int(np.ceil(np.log2(U)))
    for n in range(N + 1):
        Tg = h.level(q, "T", n).cpu().numpy()
        Tr = oracle.frame_level(e, s, q, "T", n)
        assert Tg.shape == Tr.shape
        live = np.array([[t_live(n, x, k) for k in range(Tg.shape[1])] for x in range(Tg.shape[0])])
        assert np.all(np.isnan(Tg[~live]))
        if live.any():
            assert np.max(np.abs(Tg[live] - Tr[live])) <= 2e-5 * max(1.0, np.max(np.abs(Tr))), (q, n)
    for n in range(N):
        Rg = h.level(q, "R", n).cpu().numpy()
        Rr = oracle.frame_level(e, s, q, "R", n)
        assert np.all(np.isnan(Rg[0]))
        assert np.max(np.abs(Rg[1:] - Rr[1:])) <= 2e-5 * max(1.0, np.max(np.abs(Rr))), (q, n)


@pytest.mark.parametrize("name", ["fog512", "volumetric1024", "fog2048"])
def test_forward_full_size_workloads(name):
    """The 512^2, 1024^2 and 2048^2 three-channel workloads at full size, in
    the launch configuration the autotuner picks (as the benchmark runs)."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = scenes.scene_by_name(name)
    C, H, W = e.shape
    h = HRC(W, H, C)
    h.autotune()
    F = h.forward(to_dev(e), to_dev(s)).cpu().numpy()
    h.sync()
    assert_fp32(F, oracle.fluence(e, s))


@pytest.mark.parametrize("W,H", [(70, 50), (64, 48)])
def test_forward_host_entry_matches_device_entry(W, H):
    """Host buffers, pinned or pageable, staged through device copies: the
    fluence equals the device entry point's exactly, and a backward after it
    equals the oracle's."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = scenes.random_scene(W, H, 3, 13)
    h = HRC(W, H, 3)
    Fd = h.forward(to_dev(e), to_dev(s)).cpu()
    gF = scenes.rng(14).normal(size=e.shape).astype(np.float32)
    ge_r, gs_r = oracle.fluence_adjoint(e, s, gF)
    for pinned in (True, False):
        et, st = torch.from_numpy(e.copy()), torch.from_numpy(s.copy())
        if pinned:
            et, st = et.pin_memory(), st.pin_memory()
        out = torch.empty((3, H, W), dtype=torch.float32, pin_memory=pinned)
        Fh = h.forward_host(et, st, out)
        assert torch.equal(Fd, Fh), pinned
        ge, gs = h.backward(to_dev(gF))
        assert err_max(ge.cpu().numpy(), ge_r) <= 1e-4 and err_max(gs.cpu().numpy(), gs_r) <= 1e-4


def test_autotune_keeps_results():
    """Every launch configuration the autotuner may choose gives the same
    fluence."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC, _lib
    e, s = scenes.random_scene(300, 260, 3, 14)
    h = HRC(300, 260, 3)
    ref = h.forward(to_dev(e), to_dev(s)).clone()
    for sched in (0, 1, 2):
        _lib.hrc_set_schedule(h.ctx, sched)
        F = h.forward(to_dev(e), to_dev(s))
        assert torch.equal(F, ref)
        _lib.hrc_set_timing(h.ctx, True)          # direct launches (schedule 2 runs level-major)
        F = h.forward(to_dev(e), to_dev(s))
        _lib.hrc_set_timing(h.ctx, False)
        assert torch.equal(F, ref)
    ms = h.autotune()
    assert ms > 0
    F = h.forward(to_dev(e), to_dev(s))
    assert torch.equal(F, ref)
    assert_fp32(F.cpu().numpy(), oracle.fluence(e, s))


def test_launch_configurations_give_the_same_results():
    """Every launch configuration (schedule, merge-up groups, block width, grid
    order) computes the same forward and backward: the arithmetic of each
    entry does not depend on how the work is cut into blocks."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = scenes.random_scene(70, 53, 3, 31)
    gF = scenes.rng(32).normal(size=e.shape).astype(np.float32)
    h = HRC(70, 53, 3)
    ed, sd, gd = to_dev(e), to_dev(s), to_dev(gF)
    ref = None
    for sched in (0, 1, 2):
        for groups in (1, 2, 4):
            for threads in (64, 128, 256, 512):
                for vmajor, mdown in ((0, 0), (1, 0), (0, 1), (1, 1), (0, 2), (1, 2)):
                    if mdown == 2 and sched == 2:
                        continue                  # the persistent merge down runs on one branch only
                    h.set_launch_config(sched, groups, threads, vmajor, mdown)
                    assert h.launch_config == dict(schedule=sched, groups=groups, threads=threads, vmajor=vmajor,
                                                   mdown=mdown)
                    F = h.forward(ed, sd).cpu().numpy()
                    ge, gs = h.backward(gd)
                    out = (F, ge.cpu().numpy(), gs.cpu().numpy())
                    if ref is None:
                        ref = out
                        continue
                    h.sync()
                    for a, b in zip(out, ref):
                        assert np.max(np.abs(a - b)) <= 1e-6 * max(1.0, np.max(np.abs(b))), (sched, groups, threads,
                                                                                              vmajor, mdown)


def test_bulk_copy_wait_times_out_and_recovers():
    """The bulk-copy merge down waits on a barrier with a time limit: armed
    (test hook) with bytes that never arrive, its waits give up after 1 ms,
    hrc_sync reports HRC_ETIMEOUT, and the context then computes correctly."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC, _lib
    e, s = scenes.random_scene(64, 48, 2, 51)
    h = HRC(64, 48, 2)
    h.set_launch_config(0, 1, 128, 1, 1)
    ed, sd = to_dev(e), to_dev(s)
    other = HRC(64, 48, 2)                       # a second context on the same GPU
    _lib.hrc_debug_bulk_wait(h.ctx, 16, 1_000_000)
    h.forward(ed, sd)
    Fo = other.forward(ed, sd)
    other.sync()                                 # its status word is its own: no timeout reported here
    with pytest.raises(_lib.HRCError) as ex:
        h.sync()
    assert ex.value.status == _lib.HRC_ETIMEOUT
    _lib.hrc_debug_bulk_wait(h.ctx, 0, 0)
    F = h.forward(ed, sd)
    h.sync()
    assert_fp32(F.cpu().numpy(), oracle.fluence(e, s))
    assert_fp32(Fo.cpu().numpy(), oracle.fluence(e, s))


@pytest.mark.parametrize("W,H,C,casc,seed", [
    (48, 40, 2, 0, 12), (300, 260, 3, 0, 33), (257, 130, 1, 0, 34), (1, 6, 1, 0, 35), (5, 7, 4, 0, 36),
    (64, 64, 1, 3, 37), (1030, 20, 3, 0, 38),
])
def test_persistent_merge_down_matches_bulk_and_oracle(W, H, C, casc, seed):
    """The merge down of every level in one persistent launch (mdown 2) does
    each entry's arithmetic in the same order as the one-launch-per-level
    bulk-staged kernel (mdown 1): the fluence is identical bit for bit, and
    every R level matches the oracle."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = scenes.random_scene(W, H, C, seed)
    h = HRC(W, H, C, casc)
    ed, sd = to_dev(e), to_dev(s)
    h.set_launch_config(0, 1, 128, 0, 1)
    Fb = h.forward(ed, sd).clone()
    for sched in (0, 1):
        h.set_launch_config(sched, 1, 128, 0, 2)
        F = h.forward(ed, sd)
        h.sync()
        assert torch.equal(F, Fb), sched
    assert_fp32(F.cpu().numpy(), oracle.fluence(e, s, casc))
    for q in range(4):
        U = W if q < 2 else H
        N = int(np.ceil(np.log2(U))) if U > 1 else 0
        if casc > 0:
            N = min(N, casc)
        for n in range(1, N):
            Rg = h.level(q, "R", n).cpu().numpy()
            Rr = oracle.frame_level(e, s, q, "R", n, casc)
            assert np.max(np.abs(Rg[1:] - Rr[1:])) <= 2e-5 * max(1.0, np.max(np.abs(Rr))), (q, n)


def test_persistent_merge_down_wait_times_out_and_recovers():
    """The persistent merge down bounds every dependency wait: with the test
    hook on, no item is published, so every wait on the level above gives up
    after 1 ms; hrc_sync reports HRC_ETIMEOUT and the context then computes
    correctly."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC, _lib
    e, s = scenes.random_scene(64, 48, 2, 52)
    h = HRC(64, 48, 2)
    h.set_launch_config(0, 1, 128, 0, 2)
    ed, sd = to_dev(e), to_dev(s)
    _lib.hrc_debug_bulk_wait(h.ctx, 16, 1_000_000)
    h.forward(ed, sd)
    with pytest.raises(_lib.HRCError) as ex:
        h.sync()
    assert ex.value.status == _lib.HRC_ETIMEOUT
    _lib.hrc_debug_bulk_wait(h.ctx, 0, 0)
    F = h.forward(ed, sd)
    h.sync()
    assert_fp32(F.cpu().numpy(), oracle.fluence(e, s))


def test_graph_cache_launches_directly_when_pointers_move():
    """Outputs at a new address on every call: the first six passes are
    captured, then (six cached graphs never replayed) new pointer sets run
    as direct launches; a cached set is replayed, a recurring new set is
    captured after all.  Every output is the same fluence."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC, _lib
    e, s = scenes.random_scene(64, 48, 2, 53)
    h = HRC(64, 48, 2)
    ed, sd = to_dev(e), to_dev(s)
    outs = [torch.full((2, 48, 64), float("nan"), device="cuda") for _ in range(24)]
    for o in outs:
        h.forward(ed, sd, o)
    h.sync()
    assert _lib.hrc_graph_captures(h.ctx) == 6
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    assert_fp32(outs[0].cpu().numpy(), oracle.fluence(e, s))
    h.forward(ed, sd, outs[0])                   # cached: replayed
    assert _lib.hrc_graph_captures(h.ctx) == 6
    h.forward(ed, sd, outs[20])                  # launched directly before, seen again: captured
    h.forward(ed, sd, outs[20])
    h.sync()
    assert _lib.hrc_graph_captures(h.ctx) == 7
    assert torch.equal(outs[20], outs[1])


@pytest.mark.parametrize("W,H", [(16384, 24), (24, 16384)])
def test_maximum_extent_forward_and_backward(W, H):
    """The largest accepted extent along one axis (16384: 14 cascades in the
    frames that run along it, 5 in the others): forward and backward against
    the oracle, and 16385 rejected."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC, _lib
    e, s = scenes.random_scene(W, H, 1, 90)
    gF = scenes.rng(91).normal(size=e.shape).astype(np.float32)
    h = HRC(W, H, 1)
    F = h.forward(to_dev(e), to_dev(s))
    ge, gs = h.backward(to_dev(gF))
    h.sync()
    assert_fp32(F.cpu().numpy(), oracle.fluence(e, s))
    ge_r, gs_r = oracle.fluence_adjoint(e, s, gF)
    assert err_max(ge.cpu().numpy(), ge_r) <= 1e-4
    assert err_max(gs.cpu().numpy(), gs_r) <= 1e-4
    h.close()
    with pytest.raises(_lib.HRCError) as ex:
        HRC(W + 1 if W > H else W, H + 1 if H > W else H, 1)
    assert ex.value.status == _lib.HRC_EINVAL
