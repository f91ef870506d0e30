"""Host-side logic that needs no GPU: the autotuner's cache, the seeded input
generators the tests and the benchmark share, and the approximate-space
scratch sizes of the C ABI (host-only queries)."""
import json

import numpy as np
import pytest

import synth


def test_autotune_cache_hit_skips_timing(tmp_path):
    from paper_2401_09703_gb300 import autotune
    path = tmp_path / "tune.json"
    key = autotune.cache_key("sig")
    path.write_text(json.dumps({key: {"concurrency": 16, "jacobi_block": 8, "timings": {"16x8": 1.0}}}))
    called = []
    conc, blk, timings = autotune.tune(lambda b: called.append(b), lambda hs, r: [], "sig", cache_path=str(path))
    assert (conc, blk) == (16, 8) and timings == {"16x8": 1.0}
    assert not called


def test_autotune_cache_ignores_unreadable_file(tmp_path):
    from paper_2401_09703_gb300 import autotune
    path = tmp_path / "bad.json"
    path.write_text("{not json")
    assert autotune.load_cache(str(path)) == {}
    assert autotune.load_cache(None) == {}


def test_generators_are_seeded_and_deterministic():
    a = synth.c5_problem(N=1500, k=8, s=16, n_loss=100, power_iters=1)
    b = synth.c5_problem(N=1500, k=8, s=16, n_loss=100, power_iters=1)
    assert np.array_equal(a["cols"].indices, b["cols"].indices)
    assert np.array_equal(a["S_rows"], b["S_rows"])
    assert np.allclose(a["U"], b["U"])


def test_distinct_nonempty_rows_drops_empty_and_repeated_vectors():
    r = np.array([0, 0, 2, 2, 3, 4])
    c = np.array([1, 5, 1, 5, 7, 2])
    v = np.ones(6)
    b = synth.csr_from_coo(r, c, v, 5, 10)          # rows 0 and 2 equal, row 1 empty
    out = synth.distinct_nonempty_rows(b)
    assert out.rows == 3
    dense = out.dense()
    assert dense.shape == (3, 10)
    assert not np.any(np.all(dense == 0, axis=1))
    assert len({tuple(row) for row in dense}) == 3


def test_approx_scratch_size_is_host_only():
    """svlcov_approx_work_bytes needs a handle; the workspace query for a
    descriptor with the re-orthonormalisation on grows by the Gram scratch."""
    import ctypes as C
    from paper_2401_09703_gb300 import _abi
    lib = _abi.lib()
    d = _abi.svlcov_init_desc()
    d.m, d.n, d.k, d.max_m, d.max_n, d.max_s, d.max_nnz = 100, 80, 8, 200, 200, 16, 64
    d.storage, d.small = _abi.SVLCOV_BF16, _abi.SVLCOV_SMALL_MIXED
    d.reorth = -1
    off = lib.svlcov_workspace_bytes(C.byref(d))
    d.reorth = 0       # default: on for BF16 storage
    on = lib.svlcov_workspace_bytes(C.byref(d))
    assert on > off > 0
    d.small = _abi.SVLCOV_SMALL_FP32
    d.reorth = 1       # needs FP64 small factors
    assert lib.svlcov_workspace_bytes(C.byref(d)) == 0


def test_autotune_pick_prefers_concurrency_within_slack():
    """Graph replays of many handles: within 2% of the fastest, the higher
    concurrency wins (more independent branches); outside it, the fastest."""
    from paper_2401_09703_gb300 import autotune
    cands = [(8, 8), (8, 16), (32, 8), (64, 8), (64, 16)]
    t = {"8x8": 27.2, "8x16": 27.1, "32x8": 15.6, "64x8": 15.9, "64x16": 15.7}
    assert autotune.pick(t, cands) == (64, 16)          # 15.7 and 15.9 are within 2% of 15.6
    t2 = dict(t, **{"64x8": 17.0, "64x16": 16.5})
    assert autotune.pick(t2, cands) == (32, 8)          # the 64-lane times are 6% slower
    t3 = {"8x8": 10.0, "8x16": 12.0, "32x8": 20.0, "64x8": 20.0, "64x16": 20.0}
    assert autotune.pick(t3, cands) == (8, 8)


def test_roofline_uses_the_sweep_kernels_own_time(tmp_path, monkeypatch):
    """The roofline of the dominant kernel divides its algorithmic flops
    (sweeps x 6 n^3 per launch) by the sweep kernel's own event-timed
    duration, not by the whole SVD phase's; its traffic comes from the ncu
    record only while that record matches n and the kernel's source."""
    import bench
    prof = {"svd": (300.0, 100), "jacobi_kernel": (200.0, 100)}   # ms totals, calls
    src = tmp_path / "dense.cu"
    mk = bench.SVD_MARKERS
    src.write_text(f"other code\n{mk[0]}\nkernel v1\n{mk[1]}\nmore")
    rec = tmp_path / "rec.txt"
    rec.write_text(f"# ncu record\nn = 320\nsource_sha256 = {bench._sha256(str(src))}\n"
                   "dram_bytes_read = 700000\ndram_bytes_write = 1000\n")
    monkeypatch.setattr(bench, "SVD_SOURCE", str(src))
    monkeypatch.setattr(bench, "TRAFFIC_RECORD", str(rec))
    r = bench.roofline_svd(None, prof, "mixed", 7.0, 320)
    flops = 7.0 * 6.0 * 320 ** 3
    assert r["flops_per_launch"] == flops
    assert abs(r["ms_per_launch"] - 2.0) < 1e-12
    assert abs(r["achieved"] - round(flops / 2e-3 / 1e12, 4)) < 1e-4
    assert abs(r["frac"] - round(r["achieved"] / r["peak"], 5)) < 1e-5
    assert r["traffic"] == 701000 and r["bound"] == "alu"
    assert bench.roofline_svd(None, prof, "mixed", 7.0, 640)["traffic"] is None
    src.write_text(f"changed elsewhere\n{mk[0]}\nkernel v1\n{mk[1]}\nmore")   # outside the kernel: kept
    assert bench.roofline_svd(None, prof, "mixed", 7.0, 320)["traffic"] == 701000
    src.write_text(f"other code\n{mk[0]}\nkernel v2\n{mk[1]}\nmore")   # the kernel changed since the counters
    assert bench.roofline_svd(None, prof, "mixed", 7.0, 320)["traffic"] is None


def test_sparse_roofline_bytes():
    """Algorithmic bytes of the sparse kernels: nnz (k b_f + 8) + 4 (s + 1)
    for the gather/Gram, 2 r k b_f for the scatter and s k b_f for the
    append, with r the distinct rows the batch touches."""
    import bench
    import synth
    b = synth.CSR(np.array([0, 2, 3]), np.array([5, 7, 5]), np.ones(3), 2, 10)
    k, bf = 4, 4
    want = 3 * (k * bf + 8) + 4 * 3 + 2 * 2 * k * bf + 2 * k * bf
    assert bench.sparse_bytes([("cols", b)], k, bf) == want
    prof = {"gather_gram": (1.0, 2), "apply": (1.0, 2)}
    r = bench.roofline_sparse([("rows", b), ("cols", b)], k, bf, prof, 1000.0)
    assert abs(r["achieved"] - round(2 * want / 2e-3 / 1e9, 2)) < 1e-2 and r["bound"] == "hbm"
