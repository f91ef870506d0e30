#!/usr/bin/env python
"""Benchmark of the SV-LCOV update step on GB300.

Workload (the configuration the headline metric is quoted on): graph node
insertion on a symmetric binary Chung-Lu adjacency matrix, N = 100,000 nodes
(degree exponent 2.1, mean degree 10), rank k = 64 started from the first
half of the nodes; the other half arrives in node batches of s = 256, each an
add-rows step (edges to existing nodes) followed by an add-columns step (edges
to existing and new nodes).  One benchmark step = one node batch = 512 update
vectors; the metric is update vectors (columns and rows) per second.

Paths:
  mixed  (headline) FP32 U'/V', small steps in SVLCOV_SMALL_MIXED
  plain            FP32 U'/V', small steps in FP32 (SVLCOV_SMALL_FP32)
Both are timed with CUDA events per step on the launching stream, with the
batches resident in HBM and the L2 flushed (512 MB write) between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "sparse update cols/s at k=64 (mixed vs plain FP32 GPU); rel err vs FP64 oracle"
UNIT = "update cols/s"
WORKLOAD = ("C2 graph node insertion: Chung-Lu N=100000 (gamma 2.1, mean degree 10, binary), k=64, "
            "node batches of s=256 (add_rows then add_cols)")
GOLDEN = os.path.join(ROOT, "tests", "golden", "c2_oracle_sigma.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=0, help="timed node batches (0 = all after warm-up)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="c2", choices=["c2", "c3", "c4", "c5", "stream", "lookahead"],
                    help="c2: graph node insertion (default, the headline); c3: ratings, k=128, s=1024, BF16 vs "
                         "FP32 factors; c4: 64 matrices, batched weight updates; c5: forward + backward of one "
                         "differentiated column step; stream: single-node updates, plain vs CUDA graph; "
                         "lookahead: the look-ahead projection and the tensor-core fold at 1M x 128 alone")
    ap.add_argument("--N", type=int, default=100_000)
    ap.add_argument("--k", type=int, default=64)
    ap.add_argument("--s", type=int, default=256)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-lookahead", action="store_true", help="skip the look-ahead projection measurement")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--jacobi-block", type=int, default=0,
                    help="columns per Jacobi block of the C2/streaming handles (0: the library default)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(t: float, world: int, device=None) -> float:
    """The timed region's length as the job sees it: the slowest rank's."""
    if world <= 1:
        return t
    import torch
    tt = torch.tensor([t], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
    return float(tt.item())


def whole_job_rate(units_per_rank: int, world: int, t_max: float) -> float:
    """Units all ranks processed (weak scaling: each rank runs its own replica) / slowest time."""
    return world * units_per_rank / t_max


def problem(args):
    return synth.c2_problem(N=args.N, k=args.k, s=args.s)


def c2_steps(args, npairs):
    """Warm-up and timed node batches of a C2 run (both arms use the same)."""
    W = max(0, min(args.warmup, npairs - 1))
    K = args.steps if args.steps > 0 else npairs - W
    return W, max(1, min(K, npairs - W))


def c2_config(args, world, mean_degree):
    """The config object of a C2 line (both arms print the same)."""
    return dict(workload=WORKLOAD, global_batch=2 * args.s * world, seq_len=None,
                parallelism=f"replicas x{world}" if world > 1 else "single GPU",
                l2="flushed (512 MB write) between timed steps", mean_degree=mean_degree)


# ---------------------------------------------------------------------------
class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.p = None

    def stop(self):
        if self.p is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return dict(sm_mhz=float(np.median(sm)) if sm else None, sm_max_mhz=max(mx) if mx else None,
                    reasons=sorted(reasons), samples=len(sm))


def stage(batches, torch, dev):
    from paper_2401_09703_gb300 import DeviceCSR
    out = []
    for kind, b in batches:
        out.append((kind, DeviceCSR.from_host(b.indptr, b.indices, b.values, b.rows, b.cols, device=dev,
                                             values_dtype=torch.float32)))
    return out


JACOBI_BLOCK = 0   # --jacobi-block


def make_handle(p, torch, dev, small, max_s, max_nnz):
    from paper_2401_09703_gb300 import SVLCOV
    U = torch.as_tensor(p["U"], dtype=torch.float32, device=dev)
    V = torch.as_tensor(p["V"], dtype=torch.float32, device=dev)
    s = torch.as_tensor(p["sigma"], dtype=torch.float64, device=dev)
    N = p["N"]
    return SVLCOV(U, s, V, max_m=N + 64, max_n=N + 64, max_s=max_s, max_nnz=max_nnz, storage="fp32", small=small,
                  jacobi_block=JACOBI_BLOCK)


def run_path(p, dev_batches, torch, dev, small, W, K, flush, profile=False, clocks=None):
    """Warm-up W node batches, then K timed node batches (events per step on
    the launching stream, L2 flush between steps outside the events)."""
    from paper_2401_09703_gb300 import kernel_launches
    max_s = max(b.rows for _, b in dev_batches)
    max_nnz = max(b.nnz for _, b in dev_batches)
    h = make_handle(p, torch, dev, small, max_s, max_nnz)
    stream = torch.cuda.current_stream()
    pairs = [(dev_batches[2 * i], dev_batches[2 * i + 1]) for i in range(len(dev_batches) // 2)]
    for (kr, br), (kc, bc) in pairs[:W]:
        h.add_rows(br); h.add_cols(bc)
    torch.cuda.synchronize()
    if profile:
        h.profile(True)
        h.profile_read(reset=True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    units = 0
    if clocks:
        clocks.start()
    if torch.distributed.is_initialized():
        torch.distributed.barrier()
    torch.cuda.synchronize()
    l0 = kernel_launches()
    t0 = time.perf_counter()
    for i, ((kr, br), (kc, bc)) in enumerate(pairs[W:W + K]):
        flush.zero_()
        evs[i][0].record(stream)
        h.add_rows(br)
        h.add_cols(bc)
        evs[i][1].record(stream)
        units += br.rows + bc.rows
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    launches = kernel_launches() - l0
    ck = clocks.stop() if clocks else None
    ms = [a.elapsed_time(b) for a, b in evs[:len(pairs[W:W + K])]]
    code = h.status()
    resets = h.small_state()[3]
    prof = h.profile_read() if profile else None
    U, s, V = h.get_factors(torch.float64)
    return dict(ms=ms, units=units, wall=wall, status=code, sigma=s.cpu().numpy(), launches=launches, clocks=ck,
                profile=prof, handle=h, steps=len(ms), resets=int(resets))


def run_e2e(p, batches, torch, dev, W, K):
    """End to end through the public API with host buffers: every step copies
    its batches from pinned host memory and reads Sigma back."""
    from paper_2401_09703_gb300 import DeviceCSR
    max_s = max(b.rows for _, b in batches)
    max_nnz = max(b.nnz for _, b in batches)
    h = make_handle(p, torch, dev, "mixed", max_s, max_nnz)
    stream = torch.cuda.current_stream()
    host = []
    for kind, b in batches:
        host.append((torch.as_tensor(b.indptr.astype(np.int32)).pin_memory(),
                     torch.as_tensor(b.indices.astype(np.int32)).pin_memory(),
                     torch.as_tensor(b.values.astype(np.float32)).pin_memory(), b.rows, b.cols))
    dip = torch.empty(max_s + 1, dtype=torch.int32, device=dev)
    dix = torch.empty(max_nnz, dtype=torch.int32, device=dev)
    dvv = torch.empty(max_nnz, dtype=torch.float32, device=dev)
    dip2, dix2, dvv2 = torch.empty_like(dip), torch.empty_like(dix), torch.empty_like(dvv)
    sig_host = torch.empty(h.k, dtype=torch.float64).pin_memory()
    sig_dev = torch.empty(h.k, dtype=torch.float64, device=dev)
    from paper_2401_09703_gb300 import _abi
    import ctypes as C

    def one(i, bufs):
        ip, ix, vv, rows, cols = host[i]
        a, b2, c = bufs
        a[: ip.numel()].copy_(ip, non_blocking=True)
        b2[: ix.numel()].copy_(ix, non_blocking=True)
        c[: vv.numel()].copy_(vv, non_blocking=True)
        return DeviceCSR(a[: ip.numel()], b2[: ix.numel()], c[: vv.numel()], rows, cols), ip.numel() * 4 + ix.numel() * 4 + vv.numel() * 4

    npairs = len(batches) // 2
    for i in range(W):
        br, _ = one(2 * i, (dip, dix, dvv)); h.add_rows(br)
        bc, _ = one(2 * i + 1, (dip2, dix2, dvv2)); h.add_cols(bc)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h2d = 0
    units = 0
    e0.record(stream)
    for i in range(W, min(W + K, npairs)):
        br, nb = one(2 * i, (dip, dix, dvv)); h.add_rows(br); h2d += nb
        bc, nb = one(2 * i + 1, (dip2, dix2, dvv2)); h.add_cols(bc); h2d += nb
        _abi.check(_abi.lib().svlcov_get_factors(h.h, None, C.c_void_p(sig_dev.data_ptr()), None, _abi.SVLCOV_FP64,
                                                 C.c_void_p(stream.cuda_stream)), "get_factors")
        sig_host.copy_(sig_dev, non_blocking=True)
        units += br.rows + bc.rows
    e1.record(stream)
    torch.cuda.synchronize()
    steps = max(1, min(W + K, npairs) - W)
    t = e0.elapsed_time(e1) / 1e3
    return dict(value=units / t, unit=UNIT, h2d_bytes_per_step=int(h2d / steps), d2h_bytes_per_step=8 * h.k)


TRAFFIC_RECORD = os.path.join(ROOT, "profiles", "k_jacobi_gram_c2_n320_traffic.txt")
SVD_SOURCE = os.path.join(ROOT, "paper_2401_09703_gb300", "csrc", "dense.cu")
FP32_ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12    # 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.07 GHz


SVD_MARKERS = ("// ==== Jacobi sweep kernels: begin ====", "// ==== Jacobi sweep kernels: end ====")


def _sha256(path, markers=SVD_MARKERS):
    """sha256 of the source text strictly between the two marker lines (the
    sweep kernel and the device functions it calls), or of the whole file
    when the markers are absent."""
    import hashlib
    text = open(path, encoding="utf-8").read()
    a, b = text.find(markers[0]), text.find(markers[1])
    if a >= 0 and b > a:
        text = text[text.index("\n", a) + 1:b]
    return hashlib.sha256(text.encode("utf-8")).hexdigest()


def svd_traffic(n, ldn_note=None):
    """DRAM bytes per launch of the sweep kernel at this n from the ncu
    record under profiles/ (dram__bytes_read.sum + dram__bytes_write.sum of
    one launch), or None when there is no record for this n or the kernel's
    source file has changed since the counters were taken."""
    if not os.path.exists(TRAFFIC_RECORD):
        return None, "no ncu record"
    rec = {}
    for line in open(TRAFFIC_RECORD):
        if "=" in line and not line.lstrip().startswith("#"):
            kk, v = line.split("=", 1)
            rec[kk.strip()] = v.strip()
    if int(rec.get("n", -1)) != n:
        return None, f"ncu record is for n={rec.get('n')}"
    if rec.get("source_sha256") != _sha256(SVD_SOURCE):
        return None, "kernel source changed since the ncu record"
    return int(rec["dram_bytes_read"]) + int(rec["dram_bytes_write"]), "ncu record " + os.path.basename(TRAFFIC_RECORD)


def roofline_svd(p, prof, small, sweeps_per_launch, n):
    """The dominant kernel is the Jacobi sweep kernel of the Rayleigh-Ritz
    SVD_k of K (n = k + s).  Its algorithmic work is counted as sweeps x
    6 n^3 flop per launch (the small SVD's per-sweep cost in the step's
    algorithmic work model), over the kernel's own duration: CUDA events the
    library records on its stream right around each sweep-kernel launch
    (profile phase "jacobi_kernel"), averaged over the timed steps.  The
    peak is the FP32 ALU rate of the whole GPU from unit counts and clock."""
    ms, calls = prof["jacobi_kernel"]
    per_launch_s = ms / 1e3 / max(calls, 1)
    flops = sweeps_per_launch * 6.0 * n ** 3
    achieved = flops / per_launch_s / 1e12
    traffic, tnote = svd_traffic(n)
    svd_ms, svd_calls = prof["svd"]
    return dict(bound="alu", achieved=round(achieved, 4), peak=round(FP32_ALU_PEAK_TFLOPS, 2), unit="TFLOP/s",
                frac=round(achieved / FP32_ALU_PEAK_TFLOPS, 5), traffic=traffic, traffic_source=tnote,
                kernel="k_jacobi_gram (Rayleigh-Ritz SVD_k: FP32 sweeps)", flops_per_launch=flops,
                flop_model="sweeps x 6 n^3", ms_per_launch=per_launch_s * 1e3,
                svd_phase_ms_per_call=svd_ms / max(svd_calls, 1),
                peak_note="FP32 ALU peak derived from 152 SMs x 128 lanes x 2 x 2.07 GHz (no measured ALU peak)")


def sparse_bytes(batches, k, b_f):
    """Algorithmic HBM bytes of the sparse kernels over a list of batches:
    gather + Gram (one pass: nnz (k b_f + 8) + 4 (s + 1)), scatter
    (read-modify-write of the r touched rows: 2 r k b_f) and append (s k b_f)."""
    tot = 0
    for _, b in batches:
        r = int(np.unique(b.indices).size)
        tot += b.nnz * (k * b_f + 8) + 4 * (b.rows + 1) + 2 * r * k * b_f + b.rows * k * b_f
    return tot


def roofline_sparse(batches, k, b_f, prof, peak_gbs):
    """HBM roofline of the gather/Gram (profile phase "gather") and the apply
    phase (scatter, append, the finite check and the commit: phase "apply")
    over the timed steps, L2 flushed before each step."""
    byts = sparse_bytes(batches, k, b_f)
    t = (prof["gather_gram"][0] + prof["apply"][0]) / 1e3
    achieved = byts / t / 1e9
    return dict(bound="hbm", achieved=round(achieved, 2), peak=peak_gbs, unit="GB/s", frac=round(achieved / peak_gbs, 5),
                traffic=None, kernel="k_gather_gram + k_scatter + k_append (phases gather + apply)",
                bytes_per_step=byts / max(len(batches) // 2, 1), ms_per_step=1e3 * t / max(len(batches) // 2, 1),
                peak_note="measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)")


LOOKAHEAD_WORKLOAD = ("look-ahead projection P = X'^T E^T of 64 pending batches of 1024 update vectors in one "
                      "launch: X' = U' of the C3 rating-matrix shape (1,000,000 x k=128, > L2), Poisson(20) "
                      "distinct uniform users per vector (1.31M nonzeros); and the dense fold U = U' U'' of the "
                      "same factor on the tensor cores")


def lookahead_projection(torch, dev, peak_gbs, steps=10):
    """The gather of the update step at HBM scale: svlcov_project over 65,536
    pending update vectors against a 1M x 128 factor (BF16 and FP32 storage),
    one launch per measurement, L2 flushed (512 MB write) before each.
    Algorithmic bytes per launch: nnz (k b_f + 8) for the gathered rows and
    the (index, value) pairs, 4 (s + 1) for the row pointers, and s k 8 for
    the FP64 output P."""
    from paper_2401_09703_gb300 import SVLCOV, DeviceCSR
    E = synth.lookahead_batches()
    n_users, k = E.cols, 128
    dE = DeviceCSR.from_host(E.indptr, E.indices, E.values, E.rows, E.cols, device=dev, values_dtype=torch.float32)
    gen = torch.Generator(device=dev)
    gen.manual_seed(1006)
    U0 = torch.randn(n_users, k, device=dev, generator=gen) / np.sqrt(n_users)
    V0 = torch.randn(4096, k, device=dev, generator=gen) / 64.0
    sg = torch.linspace(10.0, 1.0, k, device=dev, dtype=torch.float64)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    out = {}
    for storage, bf in (("bf16", 2), ("fp32", 4)):
        h = SVLCOV(U0, sg, V0, max_m=n_users, max_n=4096, max_s=1, max_nnz=1, storage=storage, small="mixed",
                   reorth=-1)
        h.project(0, dE, with_c0=False)                 # warm-up
        stream = torch.cuda.current_stream()
        ms = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.project(0, dE, with_c0=False)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        byts = E.nnz * (k * bf + 8) + 4 * (E.rows + 1) + E.rows * k * 8
        t = float(np.median(ms)) / 1e3
        achieved = byts / t / 1e9
        out[storage] = dict(bound="hbm", achieved=round(achieved, 1), peak=peak_gbs, unit="GB/s",
                            frac=round(achieved / peak_gbs, 4), traffic=None, kernel="k_project",
                            bytes_per_launch=int(byts), ms_per_launch=round(t * 1e3, 4), nnz=int(E.nnz),
                            vectors=int(E.rows), status=h.status())
        # the dense fold U = U' U'' of the whole factor (tensor cores), FP32 out:
        # reads rows k b_f, writes rows k 4 bytes
        Uo = torch.empty(n_users, k, dtype=torch.float32, device=dev)
        from paper_2401_09703_gb300 import _abi
        import ctypes as C
        fold = lambda: _abi.check(_abi.lib().svlcov_get_factors(h.h, C.c_void_p(Uo.data_ptr()), None, None,  # noqa
                                                                _abi.SVLCOV_FP32, C.c_void_p(stream.cuda_stream)),
                                  "get_factors")
        fold()
        fms = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fold()
            e1.record(stream)
            torch.cuda.synchronize()
            fms.append(e0.elapsed_time(e1))
        fb = n_users * k * (bf + 4)
        ft = float(np.median(fms)) / 1e3
        out[storage + "_fold"] = dict(bound="hbm", achieved=round(fb / ft / 1e9, 1), peak=peak_gbs, unit="GB/s",
                                      frac=round(fb / ft / 1e9 / peak_gbs, 4), kernel="k_rowmul_tc (U = U' U'')",
                                      bytes_per_launch=int(fb), ms_per_launch=round(ft * 1e3, 4),
                                      tensor_flops_per_launch=2 * n_users * k * k)
        del h, Uo
    del U0, V0, flush
    torch.cuda.empty_cache()
    return dict(workload=LOOKAHEAD_WORKLOAD, l2="flushed (512 MB write) before each launch", **out)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def cpu_baseline(p, seconds):
    """The FP64 oracle (sparse method, as it stands) on the host cores over a
    bounded prefix of the same trajectory."""
    from oracle import svlcov as osv
    st = osv.State.init(p["U"], p["sigma"], p["V"])
    t0 = time.perf_counter()
    units = 0
    nb = 0
    for kind, b in p["batches"]:
        st.apply(kind, b)
        units += b.rows
        nb += 1
        if time.perf_counter() - t0 > seconds and nb % 2 == 0:
            break
    t = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0))
    return dict(value=units / t, unit=UNIT, cores=cores, kind="oracle",
                sample=f"first {nb // 2} node batches ({units} update vectors) of the same trajectory, FP64 numpy/scipy")


def main_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    p = problem(args)
    from oracle import svlcov as osv
    st = osv.State.init(p["U"], p["sigma"], p["V"])
    pairs = [(p["batches"][2 * i], p["batches"][2 * i + 1]) for i in range(len(p["batches"]) // 2)]
    W, K = c2_steps(args, len(pairs))
    for (kr, br), (kc, bc) in pairs[:W]:
        st.apply(kr, br); st.apply(kc, bc)
    budget = 150.0
    t0 = time.perf_counter()
    units, done = 0, 0
    for (kr, br), (kc, bc) in pairs[W:W + K]:
        st.apply(kr, br); st.apply(kc, bc)
        units += br.rows + bc.rows
        done += 1
        if time.perf_counter() - t0 > budget:
            break
    t = time.perf_counter() - t0
    v = units / t
    cores = len(os.sched_getaffinity(0))
    line = dict(metric=METRIC, value=v, unit=UNIT, n_gpus=args.gpus, steps=done, warmup=W,
                ms_per_step=1e3 * t / max(done, 1), higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic", impl="reference",
                config=c2_config(args, 1, p["mean_degree"]),
                cpu_baseline=dict(value=v, unit=UNIT, cores=cores, kind="oracle",
                                  sample=f"{done} node batches after {W} warm-up (bounded to {budget:.0f} s); "
                                         "the oracle runs on the host cores, the L2 setting does not apply"),
                e2e=dict(value=v, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
C4_WORKLOAD = ("C4 batched weight updates A + D E^T: 64 independent matrices, m ~ U[5k, 200k], n = m/2, "
               "k in {16,32,64,128}, s ~ U[8,128], 4 nnz per column of D and E; one step = one round of 64 updates")


def c4_handles(p, torch, dev, small, jacobi_block, only_k=None, gemm_split=0):
    """Handles for the C4 matrices with seeded random orthonormal starts made
    on the device (the update step only sees the start factors)."""
    from paper_2401_09703_gb300 import SVLCOV
    gen = torch.Generator(device=dev)
    gen.manual_seed(1004)
    hs = []
    for mat in p["mats"]:
        if only_k is not None and mat["k"] != only_k:
            continue
        m, n, k = mat["m"], mat["n"], mat["k"]
        U, _ = torch.linalg.qr(torch.randn(m, k, device=dev, generator=gen))
        V, _ = torch.linalg.qr(torch.randn(n, k, device=dev, generator=gen))
        sg = 10.0 * 0.97 ** torch.arange(k, device=dev, dtype=torch.float64)
        max_s = max(b[0].rows for _, b in mat["batches"])
        max_nnz = max(max(b[0].nnz, b[1].nnz) for _, b in mat["batches"])
        hs.append(SVLCOV(U.contiguous(), sg, V.contiguous(), max_m=m, max_n=n, max_s=max_s, max_nnz=max_nnz,
                         storage="fp32", small=small, jacobi_block=jacobi_block, gemm_split=gemm_split))
        del U, V
    return hs


def main_c4(args):
    import torch
    from paper_2401_09703_gb300 import DeviceCSR, batch_run, kernel_launches
    from paper_2401_09703_gb300 import autotune
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    p = synth.c4_problem(start="none")
    R = len(p["mats"][0]["batches"])
    W = max(1, min(args.warmup, R - 1))
    K = args.steps if args.steps > 0 else R - W
    K = max(1, min(K, R - W))
    dbat = [[(DeviceCSR.from_host(D.indptr, D.indices, D.values, D.rows, D.cols, device=dev),
              DeviceCSR.from_host(E.indptr, E.indices, E.values, E.rows, E.cols, device=dev))
             for _, (D, E) in mat["batches"]] for mat in p["mats"]]
    srows = [[b[0].rows for _, b in mat["batches"]] for mat in p["mats"]]

    def items(hs, r, sel):
        return [(h, "weights", dbat[i][r]) for h, i in zip(hs, sel)]

    def run(small, conc, blk, graph, only_k=None):
        sel = [i for i, mat in enumerate(p["mats"]) if only_k is None or mat["k"] == only_k]
        # handles run side by side (conc > 0) keep their FP64 products unsplit
        split = 0 if conc == 0 else -1
        hs = c4_handles(p, torch, dev, small, blk, only_k, split)
        for r in range(W):
            if conc == 0:
                for h, i in zip(hs, sel):
                    h.update_weights(*dbat[i][r])
            else:
                batch_run(items(hs, r, sel), conc)
        torch.cuda.synchronize()
        units = sum(srows[i][r] for i in sel for r in range(W, W + K))
        s = torch.cuda.Stream()
        g = None
        note = None
        if graph:
            try:
                g = torch.cuda.CUDAGraph()
                with torch.cuda.stream(s):
                    with torch.cuda.graph(g, stream=s):
                        for r in range(W, W + K):
                            batch_run(items(hs, r, sel), conc, stream=s)
            except Exception as e:  # graph capture is an optimisation; report and run without it
                note = f"graph capture failed: {type(e).__name__}"
                g = None
                torch.cuda.synchronize()
                hs = c4_handles(p, torch, dev, small, blk, only_k, split)
                for r in range(W):
                    batch_run(items(hs, r, sel), conc)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = kernel_launches()
        with torch.cuda.stream(s):
            e0.record(s)
            if g is not None:
                g.replay()
            else:
                for r in range(W, W + K):
                    if conc == 0:
                        for h, i in zip(hs, sel):
                            h.update_weights(*dbat[i][r], stream=s)
                    else:
                        batch_run(items(hs, r, sel), conc, stream=s)
            e1.record(s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        bad = sum(1 for h in hs if h.status() != 0)
        resets = sum(h.small_state()[3] for h in hs)
        del hs, g
        torch.cuda.empty_cache()
        return dict(value=units / (ms / 1e3), unit=UNIT, ms_per_step=ms / K, launches=kernel_launches() - l0,
                    bad_status=bad, note=note, matrices=len(sel), resets_total=int(resets))

    sig = "c4:" + ",".join(str(mat["k"]) for mat in p["mats"])

    def make_handles(blk):
        return c4_handles(p, torch, dev, "mixed", blk, None, -1)

    conc, blk, timings = autotune.tune(make_handles, lambda hs, r: items(hs, r, list(range(len(hs)))), sig,
                                       cache_path=os.environ.get("SVLCOV_AUTOTUNE_CACHE"))
    res = dict(mixed_graph=run("mixed", conc, blk, True), mixed_streams=run("mixed", conc, blk, False),
               plain_sequential=run("fp32", 0, 16, False),
               k64_mixed_graph=run("mixed", conc, blk, True, only_k=64),
               k64_plain_sequential=run("fp32", 0, 16, False, only_k=64))
    head = res["mixed_graph"]
    line = dict(metric=METRIC, value=head["value"], unit=UNIT, n_gpus=1, steps=K, warmup=W,
                ms_per_step=head["ms_per_step"], higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f32 storage, f32+f64 small steps", data="synthetic",
                config=dict(workload=C4_WORKLOAD, global_batch=None, l2="factors of all 64 matrices (~2.4 GB) exceed L2",
                            autotuned=dict(concurrency=conc, jacobi_block=blk, timings_ms=timings)),
                paths=res)
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
C3_WORKLOAD = ("C3 ratings: 1,000,000 users x 50,000 items (Zipf 1.1 item popularity, ~20 ratings per user, "
               "ratings 1..5), k=128, start on the first 500,000 users (2 power iterations), users appended by "
               "add_rows in batches of s=1024 (K = 1152^2)")
C3_GOLDEN = os.path.join(ROOT, "tests", "golden", "c3_oracle_sigma.json")


def main_c3(args):
    import torch
    from paper_2401_09703_gb300 import SVLCOV, DeviceCSR, kernel_launches
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    W = max(3, args.warmup)
    K = args.steps if args.steps > 0 else 20
    p = synth.c3_problem(n_batches=W + K, power_iters=2)
    bat = [DeviceCSR.from_host(b.indptr, b.indices, b.values, b.rows, b.cols, device=dev, values_dtype=torch.float32)
           for _, b in p["batches"]]
    m0, k = p["U"].shape
    n = p["V"].shape[0]
    max_s = max(b.rows for b in bat)
    max_nnz = max(b.nnz for b in bat)
    U0 = torch.as_tensor(p["U"], dtype=torch.float32, device=dev)
    V0 = torch.as_tensor(p["V"], dtype=torch.float32, device=dev)
    s0 = torch.as_tensor(p["sigma"], device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    golden = None
    if os.path.exists(C3_GOLDEN):
        gj = json.load(open(C3_GOLDEN))
        if len(gj["sigma_after_batch"]) >= W + K:
            golden = np.array(gj["sigma_after_batch"][W + K - 1])
    stream = torch.cuda.current_stream()

    # seeded starts of the approximate variants (inputs of the method), staged once
    gst = synth.rng(1033)
    starts = [(torch.as_tensor(gst.standard_normal(b.rows), device=dev),
               torch.as_tensor(gst.standard_normal((b.rows, 10)), device=dev)) for b in bat]

    def step(h, i, b, approx):
        if approx is None:
            h.add_rows(b)
        elif approx == "gkl":
            h.add_rows_approx(b, "gkl", 10, starts[i][0])
        else:
            h.add_rows_approx(b, "rpi", 10, starts[i][1], t=3)

    def run(storage, profile=False, clocks=None, approx=None):
        h = SVLCOV(U0, s0, V0, max_m=m0 + (W + K) * max_s + 64, max_n=n + 64, max_s=max_s, max_nnz=max_nnz,
                   storage=storage, small="mixed")
        for i, b in enumerate(bat[:W]):
            step(h, i, b, approx)
        torch.cuda.synchronize()
        if profile:
            h.profile(True)
            h.profile_read(reset=True)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        if clocks:
            clocks.start()
        l0 = kernel_launches()
        units = 0
        for i, b in enumerate(bat[W:W + K]):
            flush.zero_()
            evs[i][0].record(stream)
            step(h, W + i, b, approx)
            evs[i][1].record(stream)
            units += b.rows
        torch.cuda.synchronize()
        ck = clocks.stop() if clocks else None
        launches = kernel_launches() - l0
        ms = [a.elapsed_time(c) for a, c in evs]
        out = dict(value=units / (sum(ms) / 1e3), unit=UNIT, ms_per_step=float(np.mean(ms)), status=h.status(),
                   resets=int(h.small_state()[3]), launches=launches, clocks=ck)
        sg = h.sigma().cpu().numpy()
        if golden is not None:
            keep = golden > 1e-12 * golden[0]
            out["sigma_rel_err_vs_oracle"] = float(np.max(np.abs(sg[keep] - golden[keep]) / golden[keep]))
        if profile:
            out["profile"] = h.profile_read()
        del h
        torch.cuda.empty_cache()
        return out

    res = dict(bf16=run("bf16", clocks=Clocks(0)), fp32=run("fp32"),
               gkl_l10_bf16=run("bf16", approx="gkl"), rpi_l10_t3_bf16=run("bf16", approx="rpi"))
    for kk in ("gkl_l10_bf16", "rpi_l10_t3_bf16"):   # deviation from the exact update (the approximation)
        res[kk]["note"] = "sigma_rel_err_vs_oracle is against the exact update's oracle: the approximation error"
    prof = run("bf16", profile=True)["profile"]
    pr_n = k + max_s
    sweeps = prof["svd_sweeps"] / max(prof["svd"][1], 1)
    roof = roofline_svd(p, prof, "mixed", sweeps, pr_n)
    roof["sweeps_per_launch"] = sweeps
    cpu = None
    if not args.no_cpu:
        from oracle import svlcov as osv
        st = osv.State.init(p["U"], p["sigma"], p["V"])
        t0 = time.perf_counter()
        done = 0
        for kind, b in p["batches"]:
            st.apply(kind, b)
            done += 1
            if time.perf_counter() - t0 > args.cpu_seconds:
                break
        t = time.perf_counter() - t0
        cpu = dict(value=done * max_s / t, unit=UNIT, cores=len(os.sched_getaffinity(0)), kind="oracle",
                   sample=f"first {done} add_rows batches of the same trajectory, FP64 numpy/scipy")
    head = res["bf16"]
    phases = {kk: dict(ms_total=round(v[0], 3), calls=v[1]) for kk, v in prof.items() if kk != "svd_sweeps"}
    line = dict(metric=METRIC + " [C3: BF16 vs FP32 factors]", value=head["value"], unit=UNIT, n_gpus=1, steps=K,
                warmup=W, ms_per_step=head["ms_per_step"], higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="bf16 storage, f32+f64 small steps", data="synthetic",
                config=dict(workload=C3_WORKLOAD, global_batch=max_s, l2="flushed (512 MB write) between steps"),
                paths=res, roofline=roof, phases_ms=phases, cpu_baseline=cpu, gpu_launches=int(head["launches"]),
                clocks=head["clocks"])
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
C5_WORKLOAD = ("C5 differentiated column step: C2's first node batch (Chung-Lu N=100000, k=64; the add_rows step "
               "first, untimed), then add_cols with its distinct non-empty update vectors (194 of s=256) "
               "differentiated for L = sum over 4096 existing nodes of ||U_new[r] Theta^1/2||^2; "
               "one step = forward + backward (torch autograd through the library's adjoint)")


def main_c5(args):
    import torch
    from paper_2401_09703_gb300 import SVLCOV, DeviceCSR, add_cols_with_grad, kernel_launches
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    p = synth.c5_problem()
    b, S_rows = p["cols"], p["S_rows"]
    N = p["N"]

    def to_dev(x, dtype):
        return DeviceCSR.from_host(x.indptr, x.indices, x.values, x.rows, x.cols, device=dev, values_dtype=dtype)

    def run(storage, small, W, K):
        idt = torch.float64 if storage == "fp64" else torch.float32
        h = SVLCOV(torch.as_tensor(p["U"], dtype=idt, device=dev),
                   torch.as_tensor(p["sigma"], device=dev), torch.as_tensor(p["V"], dtype=idt, device=dev),
                   max_m=N + 64, max_n=N + 64, max_s=max(b.rows, p["rows"].rows),
                   max_nnz=max(b.nnz, p["rows"].nnz), storage=storage, small=small, literal_steps=1)
        h.add_rows(to_dev(p["rows"], torch.float32))
        state = h.get_state()
        S = torch.as_tensor(S_rows, dtype=torch.int32, device=dev)
        batch = to_dev(b, torch.float64)
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        stream = torch.cuda.current_stream()
        fwd, bwd, grads = [], [], None
        l0 = None
        for it in range(W + K):
            h.set_state(state)
            flush.zero_()
            v = batch.values.detach().clone().requires_grad_(True)
            bt = DeviceCSR(batch.indptr, batch.indices, v, batch.rows, batch.cols)
            torch.cuda.synchronize()
            if it == W:
                l0 = kernel_launches()
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            U_S, th = add_cols_with_grad(h, bt, S)
            L = (U_S * U_S * th).sum()
            e1.record(stream)
            (gv,) = torch.autograd.grad(L, v)
            e2.record(stream)
            torch.cuda.synchronize()
            if it >= W:
                fwd.append(e0.elapsed_time(e1)); bwd.append(e1.elapsed_time(e2))
            grads = gv
        launches = kernel_launches() - l0
        code = h.status()
        return dict(fwd_ms=float(np.mean(fwd)), bwd_ms=float(np.mean(bwd)), steps=K, status=code,
                    launches_per_step=launches / K, grad=grads.cpu().numpy())

    W = max(3, args.warmup)
    K = args.steps if args.steps > 0 else 20
    res = {"fp32_mixed": run("fp32", "mixed", W, K), "fp64_fp64": run("fp64", "fp64", W, K)}
    head = res["fp32_mixed"]
    t = (head["fwd_ms"] + head["bwd_ms"]) / 1e3
    cpu = None
    if not args.no_cpu:
        # the oracle gradient from the oracle's own row step (cpu_baseline leg)
        from oracle import backward, svlcov as osv
        t0 = time.perf_counter()
        st = osv.State.init(p["U"], p["sigma"], p["V"])
        st.apply("rows", p["rows"])
        U, sg, V = st.factors()
        t1 = time.perf_counter()
        ga = backward.grad_autograd(U, sg, b.indptr, b.indices, b.values, b.rows, S_rows)
        t2 = time.perf_counter()
        for r in res.values():
            r["grad_rel_err_vs_oracle"] = float(np.linalg.norm(r["grad"] - ga) / np.linalg.norm(ga))
        cpu = dict(value=b.rows / (t2 - t1), unit="differentiated update cols/s", cores=len(os.sched_getaffinity(0)),
                   kind="oracle", sample="one forward + backward of the same column step (torch float64 autograd "
                                         "of the dense step); the oracle's row step before it is not timed")
    for r in res.values():
        r.pop("grad")
    line = dict(metric=METRIC + " [C5: forward + backward]", value=b.rows / t, unit="differentiated update cols/s",
                n_gpus=1, steps=K, warmup=W, ms_per_step=t * 1e3, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f32 storage, f32+f64 small steps, f64 adjoint", data="synthetic",
                config=dict(workload=C5_WORKLOAD, global_batch=b.rows, l2="flushed (512 MB write) between steps",
                            nnz=b.nnz, loss_rows=len(S_rows)),
                paths=res, cpu_baseline=cpu, gpu_launches=int(round(head["launches_per_step"] * K)))
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
STREAM_WORKLOAD = ("streaming node insertion: the C2 graph (Chung-Lu N=100000, k=64) with node batches of s=1 "
                   "(add_rows then add_cols per node, K 65^2); plain launches vs the same steps captured in one "
                   "CUDA graph")


def main_stream(args):
    import torch
    from paper_2401_09703_gb300 import DeviceCSR, kernel_launches
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    W = max(3, args.warmup)
    K = args.steps if args.steps > 0 else 400
    p = synth.c2_problem(s=1, n_batches=W + K)
    bat = [(kind, DeviceCSR.from_host(b.indptr, b.indices, b.values, b.rows, b.cols, device=dev,
                                      values_dtype=torch.float32)) for kind, b in p["batches"]]
    max_nnz = max(b.nnz for _, b in bat)

    def run(graph):
        h = make_handle(p, torch, dev, "mixed", 1, max(max_nnz, 1))
        for kind, b in bat[:2 * W]:
            h.apply(kind, b)
        torch.cuda.synchronize()
        s = torch.cuda.Stream()
        g = None
        if graph:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.stream(s):
                with torch.cuda.graph(g, stream=s):
                    for kind, b in bat[2 * W:]:
                        h.apply(kind, b, stream=s)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = kernel_launches()
        with torch.cuda.stream(s):
            e0.record(s)
            if g is not None:
                g.replay()
            else:
                for kind, b in bat[2 * W:]:
                    h.apply(kind, b, stream=s)
            e1.record(s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        updates = 2 * K
        out = dict(value=updates / (ms / 1e3), unit="updates/s", us_per_update=1e3 * ms / updates,
                   status=h.status(), launches_per_update=(kernel_launches() - l0) / updates if not graph else None,
                   sigma=h.sigma().cpu().numpy())
        return out

    res = dict(plain=run(False), graph=run(True))
    same = bool(np.array_equal(res["plain"]["sigma"], res["graph"]["sigma"]))
    cpu = None
    if not args.no_cpu:
        from oracle import svlcov as osv
        st = osv.State.init(p["U"], p["sigma"], p["V"])
        t0 = time.perf_counter()
        done = 0
        for kind, b in p["batches"]:
            st.apply(kind, b)
            done += 1
            if time.perf_counter() - t0 > args.cpu_seconds:
                break
        t = time.perf_counter() - t0
        cpu = dict(value=done / t, unit="updates/s", cores=len(os.sched_getaffinity(0)), kind="oracle",
                   sample=f"first {done} single-node updates of the same sequence, FP64 numpy/scipy")
        if done == len(p["batches"]):
            so = st.sigma
            keep = so > 1e-12 * so[0]
            res["graph"]["sigma_rel_err_vs_oracle"] = float(np.max(np.abs(res["graph"]["sigma"][keep] - so[keep])
                                                                  / so[keep]))
    for r in res.values():
        r.pop("sigma")
    head = res["graph"]
    line = dict(metric=METRIC + " [streaming, s=1]", value=head["value"], unit="updates/s", n_gpus=1, steps=K,
                warmup=W, ms_per_step=head["us_per_update"] * 2 / 1e3, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f32 storage, f32+f64 small steps", data="synthetic",
                config=dict(workload=STREAM_WORKLOAD, global_batch=2, l2="factors resident (streaming)"),
                paths=res, graph_equals_plain_bitwise=same, cpu_baseline=cpu)
    print(json.dumps(line))
    return 0


def main():
    global JACOBI_BLOCK
    args = parse()
    JACOBI_BLOCK = args.jacobi_block
    if args.impl == "reference":
        return main_reference(args)
    if args.workload == "c4":
        return main_c4(args)
    if args.workload == "c5":
        return main_c5(args)
    if args.workload == "c3":
        return main_c3(args)
    if args.workload == "stream":
        return main_stream(args)
    if args.workload == "lookahead":
        import torch
        torch.cuda.set_device(0)
        peak_gbs, peak_kind = measured_peaks()
        res = lookahead_projection(torch, torch.device("cuda", 0), peak_gbs, steps=max(3, args.steps or 10))
        print(json.dumps(dict(metric="look-ahead projection and tensor-core fold GB/s", peak_kind=peak_kind, **res)))
        return 0
    import torch
    rank, world, local = dist_env()
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    p = problem(args)
    npairs = len(p["batches"]) // 2
    W, K = c2_steps(args, npairs)
    dev_batches = stage(p["batches"], torch, dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()

    mixed = run_path(p, dev_batches, torch, dev, "mixed", W, K, flush, clocks=Clocks(local))
    t_mixed = sum(mixed["ms"]) / 1e3
    plain = None
    if not args.no_plain:
        plain = run_path(p, dev_batches, torch, dev, "fp32", W, K, flush)
    prof = run_path(p, dev_batches, torch, dev, "mixed", W, K, flush, profile=True)
    e2e = run_e2e(p, p["batches"], torch, dev, W, K)

    # max over ranks of the timed device time
    t_max = max_over_ranks(t_mixed, world, dev)
    value = whole_job_rate(mixed["units"], world, t_max)

    # accuracy against the stored FP64 oracle trajectory, after the node batch where the run stops
    err = dict(mixed=None, plain=None)
    default_shape = args.N == 100_000 and args.k == 64 and args.s == 256
    if default_shape and os.path.exists(GOLDEN):
        per = json.load(open(GOLDEN))["sigma_after_node_batch"]
        if W + K <= len(per):
            so = np.array(per[W + K - 1])
            keep = so > 1e-12 * so[0]
            err["mixed"] = float(np.max(np.abs(mixed["sigma"][keep] - so[keep]) / so[keep]))
            if plain is not None:
                err["plain"] = float(np.max(np.abs(plain["sigma"][keep] - so[keep]) / so[keep]))

    line = None
    if rank == 0:
        n = args.k + args.s
        pr = prof["profile"]
        sweeps = pr["svd_sweeps"] / max(pr["svd"][1], 1)     # average Jacobi sweeps per SVD launch
        roof = roofline_svd(p, pr, "mixed", sweeps, n)
        roof["sweeps_per_launch"] = sweeps
        peak_gbs, peak_kind = measured_peaks()
        roof_hbm = roofline_sparse(p["batches"][2 * W:2 * (W + K)], args.k, 4, pr, peak_gbs)
        roof_hbm["peak_note"] += f" ({peak_kind})"
        cpu = None if args.no_cpu else cpu_baseline(p, args.cpu_seconds)
        lookahead = None if args.no_lookahead else lookahead_projection(torch, dev, peak_gbs)
        phases = {k: dict(ms_total=round(v[0], 3), calls=v[1]) for k, v in prof["profile"].items()
                  if k != "svd_sweeps"}
        line = dict(
            metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=K, warmup=W,
            ms_per_step=1e3 * t_max / K, higher_is_better=True, scaling="weak", vs_baseline=None,
            dtype="f32 storage, f32+f64 small steps", data="synthetic",
            config=c2_config(args, world, p["mean_degree"]),
            plain_fp32=None if plain is None else dict(value=plain["units"] / (sum(plain["ms"]) / 1e3), unit=UNIT,
                                                       ms_per_step=sum(plain["ms"]) / len(plain["ms"]),
                                                       sigma_rel_err_vs_oracle=err["plain"], status=plain["status"]),
            sigma_rel_err_vs_oracle=err["mixed"], sigma_compared_after_node_batch=W + K,
            status=mixed["status"], resets=mixed["resets"],
            roofline=roof, roofline_hbm=roof_hbm, roofline_lookahead=lookahead, phases_ms=phases, e2e=e2e, cpu_baseline=cpu,
            gpu_launches=int(mixed["launches"]), clocks=mixed["clocks"],
            wall_s_timed_region=mixed["wall"])
        print(json.dumps(line))
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
