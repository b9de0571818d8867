"""Benchmark of the muffin-tin H+S generator (one JSON line on rank 0).

Metric: seconds per k-point to build H and S (and the effective TFLOP/s of
that build), split-precision form vs the FP64 form, on one GB300, at the
metric's accuracy (relative Frobenius error <= 1e-11).

A step is one pass of the whole path (radial factors, A/B coefficients,
X = T W, the H/S contraction) for one k-point of the chosen workload; inputs
are resident in HBM before the timed region. Default workload: 256 atoms of
4 species, l_max 10, N_G 20000 (H and S 6.4 GB each). Before the warm-up,
hsgen_autotune (untimed) picks the split form (slices or moduli, by the
error it measures against a 7-slice build and by time) and the schedule for
--target (default 1e-11). The timed region uses CUDA events on the
launching stream after W warm-up steps; the working set (W, X and the
operand planes, tens of GB) is far larger than the 129 MB L2, so no flush
is needed between steps.

After the timed region (not timed): `error`, whole columns of the timed H
and S against the oracle (relative Frobenius and largest per-entry error);
`fp64_form`, one timed build of the plain FP64 form on the same workload
with its own error (--no-fp64-compare skips it: about 3 minutes); `e2e`,
the same build through the C ABI from and to pinned host memory;
`cpu_baseline`, the oracle on a bounded sample.

Multi-GPU (torchrun): a multi-k-point workload deals its k-points
round-robin; a single k-point is split 2-D block-cyclically over the ranks
(hsgen_build_HS_blocks, strong scaling; --replicas: every rank builds the
whole k-point, weak scaling). No data-path collective; the barrier and the
max over ranks are only for timing.

--impl reference times the oracle (plain FP64 CPU code) on the host cores on
a bounded sample of the same workload, extrapolated to one k-point.

Other lines (not the headline): --s-form legendre (S in the m-summed
Legendre form), --l-nonsph L (T's non-spherical part up to L), --config 3
(48 k-points in one batched call), --form fp64 (the FP64 form),
--library-bars (cuBLAS FP64 / FP64-emulated products on the same operands),
--reduce (the hand-off to the generalized eigensolver on the built H, S).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H+S build s/k-pt & eff TFLOP/s: split-prec vs FP64 on 1 GB300 @<=1e-11 err"
SCHEMES = {"auto": 0, "slices": 1, "moduli": 2}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.idx)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            try:
                pw.append(float(f[3]))
            except ValueError:
                pass
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
               "samples": len(sm)}
        if pw:
            out["power_w"] = statistics.median(pw)
        return out


def _traffic(config: int, st: dict):
    """DRAM bytes per H/S depth-segment launch of the moduli kernel from the
    committed ncu record, or None when the record is for another workload,
    schedule or form, or the kernel's source has changed since."""
    import hashlib

    here = os.path.dirname(os.path.abspath(__file__))
    try:
        with open(os.path.join(here, "profiles", "crt_gemm_dram_traffic_256atoms_NG20000.json")) as f:
            rec = json.load(f)
        with open(os.path.join(here, "paper_1602_06589_gb300", "csrc", "split.cu")) as f:
            src = f.read()
    except OSError:
        return None
    try:
        a = src.index("template <int KPS_, int NST_, int CKB_>")
        b = src.index("// ---------------------------------------------------------------------------\n// Slicing kernel")
    except ValueError:
        return None
    sha = hashlib.sha256(src[a:b].encode()).hexdigest()
    if config != 4 or st.get("scheme") != 2:
        return None
    for r in (rec if isinstance(rec, list) else [rec]):  # one record per schedule captured
        if r.get("kernel_source_sha256") == sha and all(
                st.get(k) == r.get(k) for k in ("kseg_blocks", "tile_band", "unit_order", "l2_hint", "moduli")):
            return r["dram_bytes_read"] + r["dram_bytes_write"], r["algorithmic_bytes"]
    return None


# whole columns of the triangle compared with the oracle after the timed
# region: tile (64 / 128 columns) and band (1024 columns) edges, an interior
# column and the last one (the ragged tail); every row block is covered
ERROR_COLS = (0, 127, 1024, 10111, -1)


def error_columns(n):
    return sorted({c % n for c in ERROR_COLS if -n <= c < n})


def oracle_columns(system, kvec, cols):
    """The oracle's whole columns of H and S, with the per-entry scales."""
    import oracle

    t0 = time.perf_counter()
    Ho, So, norms = oracle.HS_columns(system, kvec, cols, norms=True)
    return {"cols": cols, "H": Ho, "S": So, "norms": norms, "seconds": time.perf_counter() - t0}


def column_errors(Hc, Sc, ref, uplo="U"):
    """Relative Frobenius error and the largest normwise per-entry error
    |dX_ij| / (||w_i|| ||x_j||) over the written triangle of the columns."""
    import numpy as np

    wn, xn, yn = ref["norms"]
    out = {}
    for name, A, B, sc in (("H", Hc, ref["H"], xn), ("S", Sc, ref["S"], yn)):
        d2 = b2 = per = 0.0
        for k, j in enumerate(ref["cols"]):
            rows = slice(0, j + 1) if uplo == "U" else slice(j, None)
            a, b = A[rows, k], B[rows, k]
            d2 += float(np.sum(np.abs(a - b) ** 2))
            b2 += float(np.sum(np.abs(b) ** 2))
            per = max(per, float(np.max(np.abs(a - b) / (wn[rows] * sc[k]))))
        out[name] = {"rel_frobenius": (d2 / b2) ** 0.5, "max_entry_normwise": per}
    return out


def _fp64_peak():
    """Measured FP64 DMMA peak (mma.sync.m8n8k4.f64 loop on this GPU model), if recorded."""
    try:
        with open(os.path.join(ROOT, "profiles", "fp64_dmma_peak_GB300.json")) as f:
            rec = json.load(f)
        return float(rec["tflops"]), float(rec.get("sm_mhz", 0.0)) or None
    except (OSError, KeyError, ValueError):
        return None, None


def oracle_sample_time(system, kvec, m: int):
    """Oracle cost model from two bounded samples on the host cores:
    m columns with m diagonal entries (column cost), then all m^2 pairs."""
    import numpy as np

    import oracle

    n = kvec.shape[0]
    rng = np.random.default_rng(0)
    cols = np.sort(rng.choice(n, size=m, replace=False))
    t0 = time.perf_counter()
    oracle.HS_entries(system, kvec, cols, cols)
    t1 = time.perf_counter()
    r, c = np.meshgrid(cols, cols, indexing="ij")
    oracle.HS_entries(system, kvec, r.ravel(), c.ravel())
    t2 = time.perf_counter()
    c_col = (t1 - t0) / m
    c_ent = max((t2 - t1) - (t1 - t0), 1e-9) / (m * m - m)
    full = n * c_col + n * (n + 1) / 2 * c_ent
    return full, (t2 - t0), {"c_col_s": c_col, "c_entry_s": c_ent}


def workload_name(ci, w):
    s = w.system
    ngs = [k.shape[0] for k in w.kvecs]
    ng = f"{ngs[0]}" if len(set(ngs)) == 1 else f"{min(ngs)}-{max(ngs)}"
    lm = sorted({t.lmax for t in s.types})
    return (f"{s.n_atoms} atoms / {len(s.types)} species, l_max {'/'.join(map(str, lm))}, "
            f"N_G {ng}, {len(w.kvecs)} k-point(s)")


def run_reference(args, w):
    import oracle

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    oracle.load()
    kv = w.kvecs[0]
    m = args.ref_columns
    times = []
    for i in range(args.warmup + args.steps):
        full, spent, model = oracle_sample_time(w.system, kv, m)
        if i >= args.warmup:
            times.append(full)
    value = statistics.median(times)
    cores = oracle.threads()
    line = {
        "metric": METRIC, "impl": "reference", "value": value, "unit": "s/k-point", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.config, w), "form": "oracle (plain FP64 CPU)"},
        "cpu_baseline": {"value": value, "unit": "s/k-point", "cores": cores, "kind": "oracle",
                         "sample": f"{m} plane-wave columns and {m * m} H/S entries per step, "
                                   f"extrapolated to all {kv.shape[0]} columns and the full triangle"},
        "e2e": {"value": value, "unit": "s/k-point", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_batched(args, w, world, rank, local, dist):
    """Multi-k-point workload: a step builds every k-point of the batch in one
    hsgen_build_HS_batched call (grouped launch, replayed CUDA graph)."""
    import numpy as np
    import torch

    from paper_1602_06589_gb300 import flops as fl
    from paper_1602_06589_gb300 import hsgen

    from paper_1602_06589_gb300 import partition

    sysm = w.system
    nls = [sysm.types[t].nl for t in sysm.type_of_atom]
    nk = len(w.n_g)
    flops_total = sum(fl.algorithmic_flops(n, nls)["total"] for n in w.n_g)
    # k-points are dealt round-robin to the ranks (no data exchange)
    mine = partition.kpoints_of_rank(nk, rank, world)
    n_gs = [w.n_g[k] for k in mine]
    precision = hsgen.SPLIT if args.form == "split" else hsgen.FP64
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    s_form = hsgen.S_LEGENDRE if args.s_form == "legendre" else hsgen.S_CONTRACTION
    g = hsgen.Generator(sysm, device=local, precision=precision, slices=args.slices, s_form=s_form,
                        target_rel_err=args.target, scheme=SCHEMES[args.scheme], moduli=args.moduli,
                        h_form=hsgen.H_HPD if args.h_form == "hpd" else hsgen.H_TW)
    kv_host = [np.ascontiguousarray(w.kvecs[k]) for k in mine]
    Hs = [torch.zeros((n, n), dtype=torch.complex128, device=dev) for n in n_gs]
    Ss = [torch.zeros_like(h) for h in Hs]
    if precision == hsgen.SPLIT and not args.no_autotune and n_gs:
        # untimed: form and schedule tuned on the largest k-point of the batch
        kbig = int(np.argmax(n_gs))
        g.autotune(torch.from_numpy(kv_host[kbig]).to(dev), Hs[kbig], Ss[kbig])

    def step():
        hsgen.hsgen_build_HS_batched(g.ctx, n_gs, [k.ctypes.data for k in kv_host], [h.data_ptr() for h in Hs],
                                     [s.data_ptr() for s in Ss], n_gs, stream.cuda_stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    if dist:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    st = g.stats()
    line = {
        "metric": METRIC, "value": ms * 1e-3 / nk, "unit": "s/k-point", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
        "scaling": "strong", "vs_baseline": None, "dtype": "bf16-split/f64" if precision == hsgen.SPLIT else "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(args.config, w), "form": args.form, "s_form": args.s_form,
                   "k_points_per_step": nk,
                   "parallelism": f"k-points dealt round-robin over {world} rank(s)",
                   "launch": "hsgen_build_HS_batched (grouped persistent launch, CUDA graph replay)"},
        "eff_tflops": flops_total / (ms * 1e-3) / 1e12, "gpu_launches": st["kernel_launches"] * args.steps,
    }
    clk_s = clk.summary()
    if clk_s:
        line["clocks"] = clk_s
    st = g.stats()
    line["config"]["scheme"] = {1: "slices (Ozaki I)", 2: "moduli (Ozaki II)"}.get(st["scheme"])
    line["config"]["bf16_products_per_fp64_product"] = st["products"]
    if not args.no_sequential and precision == hsgen.SPLIT:
        # the same k-points as separate hsgen_build_HS calls (one k-point each, same context)
        kv_dev = [torch.from_numpy(k).to(dev) for k in kv_host]
        for k in range(len(n_gs)):
            g.build(kv_dev[k], Hs[k], Ss[k])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            for k in range(len(n_gs)):
                g.build(kv_dev[k], Hs[k], Ss[k])
        e1.record(stream)
        torch.cuda.synchronize()
        seq_ms = e0.elapsed_time(e1) / args.steps
        line["sequential"] = {"s_per_kpoint": seq_ms * 1e-3 / max(1, len(n_gs)), "ms_per_step": seq_ms,
                              "batched_speedup": seq_ms / ms,
                              "how": "one hsgen_build_HS call per k-point, same context and schedule"}
    g.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def _cublas(torch):
    """The cuBLAS library torch has loaded (the same instance, so its handle is valid)."""
    import ctypes

    a = torch.zeros((2, 2), dtype=torch.complex128, device="cuda")
    (a @ a).sum().item()  # makes torch initialise cuBLAS
    path = None
    with open("/proc/self/maps") as f:
        for line in f:
            if "libcublas.so" in line and "libcublasLt" not in line:
                path = line.split()[-1]
                break
    if path is None:
        raise RuntimeError("libcublas is not loaded")
    lib = ctypes.CDLL(path)
    vp, i = ctypes.c_void_p, ctypes.c_int
    lib.cublasZgemm_v2.argtypes = [vp, i, i, i, i, i, vp, vp, i, vp, i, vp, vp, i]
    lib.cublasZherk_v2.argtypes = [vp, i, i, i, i, vp, vp, i, vp, vp, i]
    lib.cublasDgemm_v2.argtypes = [vp, i, i, i, i, i, vp, vp, i, vp, i, vp, vp, i]
    lib.cublasSetMathMode.argtypes = [vp, i]
    lib.cublasSetEmulationStrategy.argtypes = [vp, i]
    return lib


def reduce_bench(args, w):
    """The generalized-eigenproblem hand-off (Sec. 2.3, Eq. matrix_kohnsham) on
    this workload: H, S from the split build plus a stand-in for the
    interstitial part (S + I, H + diag(|K_t|^2)), then hsgen_reduce_generalized
    (FP64 Cholesky of S and H~ = U^-H H U^-1 in place) timed with CUDA events;
    each timed call starts from a fresh device copy of H, S (copy untimed)."""
    import numpy as np
    import torch

    from paper_1602_06589_gb300 import hsgen

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    sysm, kv = w.system, w.kvecs[0]
    n = kv.shape[0]
    with hsgen.Generator(sysm, precision=hsgen.SPLIT) as g:
        # the reduction's form follows the context's precision
        gr = g if args.form == "split" else hsgen.Generator(sysm, precision=hsgen.FP64)
        H, S = g.build(torch.from_numpy(kv).to(dev))
        H += torch.diag(torch.from_numpy(np.sum(kv * kv, axis=1)).to(H)).triu()
        S += torch.eye(n, dtype=S.dtype, device=dev)
        build_s = g.stats()["ms_total"] * 1e-3
        H0, S0 = H.clone(), S.clone()
        times = []
        for i in range(max(1, args.warmup) + args.steps):
            H.copy_(H0)
            S.copy_(S0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            gr.reduce(H, S, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            if i >= max(1, args.warmup):
                times.append(e0.elapsed_time(e1) * 1e-3)
        if gr is not g:
            gr.close()
    t = statistics.median(times)
    flops = (8.0 / 3.0 + 8.0) * float(n) ** 3  # Cholesky n^3/3 + two solves n^3/2 complex MACs each, 8 flops per MAC
    peaks = _peaks()
    bf16 = peaks.get("bf16_tflops_sustained", 1700.0)
    p64, _ = _fp64_peak()
    fp64_peak = p64 or bf16 * 1.25 / 2250.0
    achieved = flops / t / 1e12
    # blocks of 128 rows: FP64 tile kernels for the diagonal blocks; products as
    # 7-slice BF16 products (28 slice pairs, split form) or FP64 DMMA (FP64 form)
    split = args.form == "split"
    line = {"metric": "generalized-eigenproblem reduction (Cholesky of S, H~ = U^-H H U^-1), s/k-point",
            "impl": "reduce", "value": t, "unit": "s/k-point", "n_gpus": 1, "steps": args.steps,
            "warmup": max(1, args.warmup), "higher_is_better": False, "dtype": "bf16-split/f64" if split else "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(args.config, w), "interstitial": "stand-in S + I, H + diag(|K|^2)",
                       "form": "split: FP64 tile kernels on the diagonal blocks, 7-slice BF16 products" if split
                       else "FP64: FP64 tile kernels on the diagonal blocks, FP64 DMMA products"},
            "build_s_per_kpoint": build_s, "fp64_equivalent_tflops": achieved,
            "roofline": ({"bound": "tensor", "achieved": flops * 28 / t / 1e12, "peak": bf16, "unit": "TFLOP/s",
                          "frac": flops * 28 / t / 1e12 / bf16, "traffic": None,
                          "kernel": "whole reduction as BF16 slice products (upper bound: FP64 diagonal blocks counted)",
                          "peak_source": "measured bf16 sustained"} if split else
                         {"bound": "tensor", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                          "frac": achieved / fp64_peak, "traffic": None,
                          "kernel": "whole reduction in FP64 (DMMA products, FP64 tile kernels)",
                          "peak_source": "measured FP64 DMMA loop" if p64 else
                                         "measured bf16 sustained x nominal fp64/bf16 ratio"})}
    print(json.dumps(line), flush=True)


def library_bars(args, w):
    """Library bars on the same workload, beside this library's split form:
    (1) cuBLAS ZGEMM (H = W^H X, full) + ZHERK (S = V^H V, V = diag(sqrt(u)) W,
    upper triangle) in plain FP64; (2) the same products in real form,
    Re/Im H = [Wr; Wi]^T [Xr; Xi] / [Wr; Wi]^T [Xi; -Xr] and likewise for S,
    as four DGEMMs of depth 2D, in plain FP64 and with cuBLAS's FP64
    fixed-point emulation (EAGER strategy). Operands are built with this
    library's coefficient and T-matrix calls; the cuBLAS calls are the library
    under test and are timed without operand construction."""
    import ctypes

    import numpy as np
    import torch

    from paper_1602_06589_gb300 import flops, hsgen

    dev = torch.device("cuda", 0)
    sysm, kv = w.system, w.kvecs[0]
    n = kv.shape[0]
    nls = [sysm.types[t].nl for t in sysm.type_of_atom]
    fa = flops.algorithmic_flops(n, nls)
    lib = _cublas(torch)
    handle = ctypes.c_void_p(torch.cuda.current_blas_handle())
    kvd = torch.from_numpy(kv).to(dev)
    with hsgen.Generator(sysm, precision=hsgen.SPLIT) as g:
        # ours: the split form, timed like the benchmark
        H1, S1 = g.build(kvd)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ours = []
        for _ in range(3):
            torch.cuda.synchronize()
            ev[0].record()
            H1, S1 = g.build(kvd, H1.mT, S1.mT)
            ev[1].record()
            torch.cuda.synchronize()
            ours.append(ev[0].elapsed_time(ev[1]) / 1e3)
        off = g.depth_offsets
        Wpad = g.coefficients(kvd).mT  # (N_G, depth): row t = column t of W
        rows, urow = [], []
        for a, ti in enumerate(sysm.type_of_atom):
            ty = sysm.types[ti]
            nl = ty.nl
            rows.append(np.arange(off[a], off[a] + 2 * nl))
            l_of = np.repeat(np.arange(ty.lmax + 1), 2 * np.arange(ty.lmax + 1) + 1)
            urow.append(np.concatenate([np.ones(nl), np.asarray(ty.udot_norm2)[l_of]]))
        rows = torch.from_numpy(np.concatenate(rows)).to(dev)
        u = torch.from_numpy(np.concatenate(urow)).to(dev)
        Wc = Wpad[:, rows].contiguous()  # (N_G, D): column-major D x N_G, ld D
        del Wpad
        D = Wc.shape[1]
        X = torch.empty_like(Wc)
        c0 = 0
        for a, ti in enumerate(sysm.type_of_atom):
            m2 = 2 * sysm.types[ti].nl
            T = torch.from_numpy(g.T_matrix(ti)).to(dev)
            X[:, c0:c0 + m2] = Wc[:, c0:c0 + m2] @ T.mT  # X_a = T W_a
            c0 += m2
        V = (Wc * torch.sqrt(u)).contiguous()
    Hc = torch.zeros((n, n), dtype=torch.complex128, device=dev)  # column-major buffers
    Sc = torch.zeros_like(Hc)
    one = (ctypes.c_double * 2)(1.0, 0.0)
    zero = (ctypes.c_double * 2)(0.0, 0.0)
    d1, d0 = ctypes.c_double(1.0), ctypes.c_double(0.0)

    def run():
        st = lib.cublasZgemm_v2(handle, 2, 0, n, n, D, ctypes.cast(one, ctypes.c_void_p), Wc.data_ptr(), D,
                                X.data_ptr(), D, ctypes.cast(zero, ctypes.c_void_p), Hc.data_ptr(), n)
        st2 = lib.cublasZherk_v2(handle, 1, 2, n, D, ctypes.byref(d1), V.data_ptr(), D, ctypes.byref(d0),
                                 Sc.data_ptr(), n)
        if st or st2:
            raise RuntimeError(f"cuBLAS status {st} {st2}")

    def timed(fn, reps):
        fn()
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            ev[0].record()
            fn()
            ev[1].record()
            torch.cuda.synchronize()
            ts.append(ev[0].elapsed_time(ev[1]) / 1e3)
        return statistics.median(ts)

    iu = torch.triu_indices(n, n, device=dev)

    def rel(A, B):  # A, B column-major buffers, compared on the upper triangle
        a, b = A.mT[iu[0], iu[1]], B.mT[iu[0], iu[1]]
        return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))

    t_native = timed(run, args.bar_reps)
    Hn, Sn = Hc.clone(), Sc.clone()
    del Hc, Sc
    # real form: stacked (n, 2D) row-major = column-major 2D x n operands
    Wr = torch.cat([Wc.real, Wc.imag], dim=1).contiguous()
    Xr = torch.cat([X.real, X.imag], dim=1).contiguous()
    Xs = torch.cat([X.imag, -X.real], dim=1).contiguous()
    Vr = torch.cat([V.real, V.imag], dim=1).contiguous()
    Vs = torch.cat([V.imag, -V.real], dim=1).contiguous()
    del Wc, X, V
    R = [torch.zeros((n, n), dtype=torch.float64, device=dev) for _ in range(4)]
    d_one, d_zero = ctypes.c_double(1.0), ctypes.c_double(0.0)

    def run_real():
        for (A, B, C) in ((Wr, Xr, R[0]), (Wr, Xs, R[1]), (Vr, Vr, R[2]), (Vr, Vs, R[3])):
            st = lib.cublasDgemm_v2(handle, 1, 0, n, n, 2 * D, ctypes.byref(d_one), A.data_ptr(), 2 * D,
                                    B.data_ptr(), 2 * D, ctypes.byref(d_zero), C.data_ptr(), n)
            if st:
                raise RuntimeError(f"cuBLAS DGEMM status {st}")

    def as_complex():
        return torch.complex(R[0], R[1]), torch.complex(R[2], R[3])

    t_real = timed(run_real, args.bar_reps)
    Hr, Sr = as_complex()
    err_real = (rel(Hr, Hn), rel(Sr, Sn))
    del Hr, Sr
    lib.cublasSetMathMode(handle, 8)  # CUBLAS_FP64_EMULATED_FIXEDPOINT_MATH
    lib.cublasSetEmulationStrategy(handle, 2)  # CUBLAS_EMULATION_STRATEGY_EAGER
    try:
        t_emul = timed(run_real, args.bar_reps)
    finally:
        lib.cublasSetMathMode(handle, 0)
        lib.cublasSetEmulationStrategy(handle, 0)
    He, Se = as_complex()
    err_emul = (rel(He, Hn), rel(Se, Sn))
    F = fa["total"]
    out = {
        "metric": METRIC, "impl": "library-bars", "unit": "s/k-point",
        "config": {"workload": workload_name(args.config, w), "depth": D},
        "ours_split": {"s": statistics.median(ours), "eff_tflops": F / statistics.median(ours) / 1e12,
                       "rel_err_H_vs_cublas_fp64": rel(H1.mT, Hn), "rel_err_S_vs_cublas_fp64": rel(S1.mT, Sn)},
        "cublas_fp64": {"s": t_native, "eff_tflops": F / t_native / 1e12, "calls": "ZGEMM (H, full) + ZHERK (S)"},
        "cublas_fp64_real_form": {"s": t_real, "eff_tflops": F / t_real / 1e12, "calls": "4 DGEMM, depth 2D",
                                  "rel_err_H": err_real[0], "rel_err_S": err_real[1]},
        "cublas_fp64_emulated": {"s": t_emul, "eff_tflops": F / t_emul / 1e12, "calls": "4 DGEMM, depth 2D",
                                 "rel_err_H": err_emul[0], "rel_err_S": err_emul[1],
                                 "mode": "CUBLAS_FP64_EMULATED_FIXEDPOINT_MATH, EAGER"},
        "note": "H + S only (operands pre-built, not timed) for cuBLAS; ours includes coefficients and T-apply",
    }
    print(json.dumps(out), flush=True)


def roofline(st, f_contract, c_ms, precision, peaks, clk_s, args, hsgen):
    """Roofline of the dominant kernel (the H/S contraction) from the library's
    own CUDA events. Split form: executed BF16 products per second against the
    measured cuBLAS BF16 GEMM peak; `frac` scales that peak to the SM clock
    sampled during this run (the peak was taken at its own median clock under
    the power cap), `frac_vs_measured_peak` is the unscaled ratio. FP64 form:
    algorithmic FP64 flops per second against the measured FP64 DMMA peak."""
    mhz = clk_s["sm_mhz"] if clk_s else None
    if precision == hsgen.SPLIT:
        scheme = st.get("scheme", 0)
        units = st.get("products", 0) or st["slices"] * (st["slices"] + 1) // 2
        lp_flops = f_contract * units  # bf16 products actually executed
        achieved = lp_flops / (c_ms * 1e-3) / 1e12
        peak = peaks.get("bf16_tflops_sustained", 1700.0)
        pmhz = (peaks.get("clocks_under_load") or {}).get("sm_mhz_median")
        peak_clk = peak * mhz / pmhz if (mhz and pmhz) else peak
        tr = _traffic(args.config, st) \
            if not args.n_g and st.get("s_form") != hsgen.S_LEGENDRE else None
        return {"bound": "tensor", "achieved": achieved, "peak": peak_clk, "unit": "TFLOP/s",
                "frac": achieved / peak_clk, "frac_vs_measured_peak": achieved / peak,
                "measured_peak": peak, "measured_peak_mhz": pmhz, "run_mhz": mhz,
                "bf16_products_per_fp64_mac": units,
                "traffic": tr[0] if tr else None,
                "traffic_unit": "DRAM bytes per H/S depth-segment launch (ncu, 1 pass)",
                "traffic_algorithmic_bytes": tr[1] if tr else None,
                "kernel": ("H/S contraction, moduli scheme (crt_gemm_kernel, tcgen05 bf16)" if scheme == 2 else
                           "H/S contraction, slices scheme (split_gemm_kernel, tcgen05 bf16)"),
                "peak_source": ("measured bf16 sustained (MEASURED_PEAKS.json), scaled to the sampled SM clock"
                                if "bf16_tflops_sustained" in peaks else "fallback")}
    achieved = f_contract / (c_ms * 1e-3) / 1e12
    p64, p64_mhz = _fp64_peak()
    if p64:
        peak = p64 * mhz / p64_mhz if (mhz and p64_mhz) else p64
        src = "measured FP64 DMMA loop (profiles/fp64_dmma_peak_GB300.json)" + (", scaled to the sampled SM clock"
                                                                              if (mhz and p64_mhz) else "")
    else:
        peak = peaks.get("bf16_tflops_sustained", 1700.0) * 1.25 / 2250.0
        src = "measured bf16 sustained x nominal fp64/bf16 ratio"
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "run_mhz": mhz, "traffic": None, "kernel": "FP64 H/S contraction (mma.sync f64)", "peak_source": src}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--form", choices=["split", "fp64"], default="split")
    ap.add_argument("--config", type=int, default=4)
    ap.add_argument("--slices", type=int, default=0)
    ap.add_argument("--moduli", type=int, default=0, help="split form, moduli scheme: moduli count (0: from the target)")
    ap.add_argument("--scheme", choices=sorted(SCHEMES), default="auto",
                    help="split form: slices (Ozaki I), moduli (Ozaki II) or auto (moduli when they meet the target)")
    ap.add_argument("--target", type=float, default=1e-11,
                    help="split form: relative error the slice or moduli count is chosen for (the metric's 1e-11)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-sequential", action="store_true",
                    help="multi-k-point workload: skip timing the k-points as separate hsgen_build_HS calls")
    ap.add_argument("--replicas", action="store_true",
                    help="several GPUs, one k-point: every rank builds the whole k-point (weak scaling) instead of "
                         "its 2-D block-cyclic blocks")
    ap.add_argument("--ref-columns", type=int, default=384)
    ap.add_argument("--n-g", type=int, default=0, help="override N_G (smaller cases for profiling)")
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="skip the FP64-form step timed after the split form on the same workload")
    ap.add_argument("--no-error", action="store_true",
                    help="skip the comparison of whole columns of H and S with the oracle")
    ap.add_argument("--l-nonsph", type=int, default=-1,
                    help="l_nonsph of every species (default: l_max, a dense T)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip hsgen_autotune before the warm-up (split form)")
    ap.add_argument("--s-form", choices=["contraction", "legendre"], default="contraction",
                    help="S as the A^H A + B^H U B contraction (default) or in the m-summed Legendre form")
    ap.add_argument("--h-form", choices=["tw", "hpd"], default="tw",
                    help="H as W^H (T W) for every species (default) or by the HPD route (Sec. 4.6.2-4.6.3: "
                         "species whose T passes the Cholesky test take Y = C^H W and H = Y^H Y)")
    ap.add_argument("--shift-energies", type=float, default=0.0,
                    help="raise every E_l of the synthetic radial data by this much (12 makes every species' "
                         "T positive definite)")
    ap.add_argument("--library-bars", action="store_true",
                    help="time cuBLAS ZGEMM + ZHERK (FP64 and FP64-emulated) beside the split form, then exit")
    ap.add_argument("--bar-reps", type=int, default=1)
    ap.add_argument("--reduce", action="store_true",
                    help="time the generalized-eigenproblem hand-off (hsgen_reduce_generalized) on this "
                         "workload, then exit")
    args = ap.parse_args()

    from workloads import make_config

    w = make_config(args.config, n_g_override=args.n_g or None)
    if args.shift_energies:
        from workloads import shift_energies

        w.system = shift_energies(w.system, args.shift_energies)
    if args.l_nonsph >= 0:  # T's non-spherical part only for l, l' <= l_nonsph (Fig. Tmat_structure)
        for ty in w.system.types:
            ty.lmax_nonsph = min(args.l_nonsph, ty.lmax)
    if args.impl == "reference":
        run_reference(args, w)
        return
    if args.library_bars:
        library_bars(args, w)
        return
    if args.reduce:
        import __graft_entry__

        __graft_entry__.build()
        reduce_bench(args, w)
        return

    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__

    if rank == 0 or world == 1:
        __graft_entry__.build()
    if dist:
        dist.barrier()
    from paper_1602_06589_gb300 import flops as fl
    from paper_1602_06589_gb300 import hsgen

    sysm = w.system
    if len(w.kvecs) > 1:
        run_batched(args, w, world, rank, local, dist)
        return
    kv_host = w.kvecs[0]
    n = kv_host.shape[0]
    nls = [sysm.types[t].nl for t in sysm.type_of_atom]
    fal = fl.algorithmic_flops(n, nls)
    precision = hsgen.SPLIT if args.form == "split" else hsgen.FP64
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    s_form = hsgen.S_LEGENDRE if args.s_form == "legendre" else hsgen.S_CONTRACTION
    g = hsgen.Generator(sysm, device=local, precision=precision, slices=args.slices, s_form=s_form,
                        target_rel_err=args.target, scheme=SCHEMES[args.scheme], moduli=args.moduli,
                        h_form=hsgen.H_HPD if args.h_form == "hpd" else hsgen.H_TW)
    kv = torch.from_numpy(kv_host).to(dev)
    H = torch.zeros((n, n), dtype=torch.complex128, device=dev)
    S = torch.zeros_like(H)
    if precision == hsgen.SPLIT and not args.no_autotune:
        g.autotune(kv, H, S)  # untimed: picks the split form, the depth segment and the tile band
    tuned = g.stats()
    # several ranks and one k-point: the k-point's H and S split 2-D
    # block-cyclically over the most square process grid (strong scaling);
    # --replicas: every rank builds the whole k-point (weak scaling)
    from paper_1602_06589_gb300 import partition

    blocks = world > 1 and not args.replicas
    prow, pcol = partition.grid_shape(world)
    myrow, mycol = divmod(rank, pcol)
    BLOCK = 256

    def build():
        if blocks:
            hsgen.hsgen_build_HS_blocks(g.ctx, n, kv.data_ptr(), H.data_ptr(), S.data_ptr(), n, BLOCK, prow, pcol,
                                        myrow, mycol, stream.cuda_stream)
        else:
            g.build(kv, H, S)

    for _ in range(args.warmup):
        build()
    torch.cuda.synchronize()
    contract_ms, launches = [], 0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            build()
            st = g.stats()  # reads the library's own events (recorded on this stream)
            contract_ms.append(st["ms_contract"])
            launches += st["kernel_launches"]
        ev1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    if dist:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    st = g.stats()
    s_per_k = ms * 1e-3 if blocks else ms * 1e-3 / world  # one k-point over all ranks, or one per rank
    eff_tflops = fal["total"] / (ms * 1e-3) / 1e12
    peaks = _peaks()

    # dominant kernel: the H/S contraction
    c_ms = statistics.mean(contract_ms) or st["ms_total"]
    # with S in the Legendre form the contraction computes H only (half of F_HS),
    # over the rows l <= l_nonsph of each atom
    if st.get("s_form") == hsgen.S_LEGENDRE:
        nlc = []
        for t in sysm.type_of_atom:
            ty = sysm.types[t]
            lc = ty.lmax if getattr(ty, "lmax_nonsph", None) is None else min(ty.lmax_nonsph, ty.lmax)
            nlc.append((lc + 1) ** 2)
        f_contract = fl.algorithmic_flops(n, nlc)["F_HS"] / 2
    else:
        f_contract = fal["F_HS"]
    clk_s = clk.summary()
    roof = roofline(st, f_contract, c_ms, precision, peaks, clk_s, args, hsgen)

    line = {
        "metric": METRIC, "value": s_per_k, "unit": "s/k-point", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
        "scaling": "strong" if blocks else "weak",
        "vs_baseline": None, "dtype": "bf16-split/f64" if precision == hsgen.SPLIT else "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(args.config, w), "form": args.form,
                   "s_form": "legendre (Eq. overlap_no_m, FP64)" if st.get("s_form") == hsgen.S_LEGENDRE
                   else "contraction",
                   "l_nonsph": args.l_nonsph if args.l_nonsph >= 0 else "l_max",
                   "h_form": ({"route": "hpd", "species_routed": st.get("hpd_species", 0)}
                              if args.h_form == "hpd" else "tw"),
                   "energy_shift": args.shift_energies,
                   "slices": st["slices"] if precision == hsgen.SPLIT else None,
                   "scheme": ({1: "slices (Ozaki I)", 2: "moduli (Ozaki II)"}.get(st["scheme"])
                              if precision == hsgen.SPLIT else None),
                   "moduli": st["moduli"] if precision == hsgen.SPLIT else None,
                   "operand_column_norm_bits": st["bits"] if precision == hsgen.SPLIT else None,
                   "bf16_products_per_fp64_product": st["products"] if precision == hsgen.SPLIT else None,
                   "target_rel_err": args.target if precision == hsgen.SPLIT else None,
                   "atom_chunks": st["atom_chunks"],
                   "schedule": ({"kseg_blocks": tuned["kseg_blocks"], "tile_band": tuned["tile_band"],
                                 "stage_geometry": tuned["stage_geometry"], "unit_order": tuned["unit_order"],
                                 "l2_hint": tuned["l2_hint"], "autotuned": not args.no_autotune,
                                 "autotune_measured_rel_err": tuned["tuned_rel_err"]}
                                if precision == hsgen.SPLIT else None),
                   "l2": "working set >> L2 (no flush needed)",
                   "parallelism": (f"one k-point, H/S blocks of {BLOCK} 2-D block-cyclic over a {prow} x {pcol} grid"
                                   if blocks else f"k-point replicas x{world}")},
        "eff_tflops": eff_tflops, "flops_per_kpoint": fal["total"],
        "phases_ms": {k: st[k] for k in ("ms_coefficients", "ms_tapply", "ms_slice", "ms_contract", "ms_s", "ms_total")},
        "roofline": roof, "gpu_launches": launches,
    }
    if clk_s:
        line["clocks"] = clk_s

    if not args.no_e2e and blocks:
        # end to end, one k-point over the grid: K_t from pinned host memory,
        # the rank's blocks built, its block columns copied to pinned host memory
        kh = torch.from_numpy(kv_host.copy()).pin_memory()
        mine = [J for J in range((n + BLOCK - 1) // BLOCK) if J % pcol == mycol]
        Hh = torch.empty((len(mine) * BLOCK, n), dtype=torch.complex128).pin_memory()
        Sh = torch.empty_like(Hh).pin_memory()
        e_steps = max(1, min(args.steps, 3))
        dist.barrier()
        t0 = time.perf_counter()
        for _ in range(e_steps):
            kv.copy_(kh, non_blocking=True)
            build()
            r0 = 0
            for J in mine:
                c0, c1 = J * BLOCK, min(n, (J + 1) * BLOCK)
                Hh[r0:r0 + c1 - c0].copy_(H[c0:c1], non_blocking=True)  # row c of the buffer = column c
                Sh[r0:r0 + c1 - c0].copy_(S[c0:c1], non_blocking=True)
                r0 += c1 - c0
            torch.cuda.synchronize()
        te = (time.perf_counter() - t0) / e_steps
        t = torch.tensor([te], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        line["e2e"] = {"value": float(t.item()), "unit": "s/k-point", "h2d_bytes_per_step": int(kh.numel() * 8),
                       "d2h_bytes_per_step": int(2 * sum(min(n, (J + 1) * BLOCK) - J * BLOCK for J in mine) * n * 16),
                       "note": "per rank: its block columns (all rows) of H and S"}
        del Hh, Sh
    elif not args.no_e2e:
        # end to end through the C ABI with host buffers (copies inside the timed region)
        kh = torch.from_numpy(kv_host.copy()).pin_memory()
        Hh = torch.empty((n, n), dtype=torch.complex128).pin_memory()
        Sh = torch.empty((n, n), dtype=torch.complex128).pin_memory()
        hsgen.hsgen_build_HS(g.ctx, n, kh.data_ptr(), Hh.data_ptr(), Sh.data_ptr(), n, stream.cuda_stream)
        if dist:
            dist.barrier()
        e_steps = max(1, min(args.steps, 3))
        walls, dev_ms, up_ms, down_ms = [], [], [], []
        t0 = time.perf_counter()
        for _ in range(e_steps):
            t1 = time.perf_counter()
            hsgen.hsgen_build_HS(g.ctx, n, kh.data_ptr(), Hh.data_ptr(), Sh.data_ptr(), n, stream.cuda_stream)
            walls.append(time.perf_counter() - t1)
            est = g.stats()
            dev_ms.append(est["ms_total"])  # the build's device time, without the copies
            up_ms.append(est["ms_upload"])
            down_ms.append(est["ms_download"])
        te = (time.perf_counter() - t0) / e_steps
        if dist:
            t = torch.tensor([te], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            te = float(t.item())
        # after the timed calls: this box's device-to-pinned-host copy rate (one
        # 6.4 GB copy of H), which bounds how fast the copy-out can keep pace
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        Hh.copy_(H, non_blocking=True)
        c1.record(stream)
        c1.synchronize()
        d2h = H.numel() * 16 / (c0.elapsed_time(c1) * 1e-3) / 1e9
        line["e2e"] = {"value": te / world, "unit": "s/k-point", "h2d_bytes_per_step": int(kh.numel() * 8),
                       "d2h_bytes_per_step": int(2 * n * n * 16),
                       "calls_s": [round(x, 4) for x in walls], "device_ms": [round(x, 1) for x in dev_ms],
                       "upload_ms": [round(x, 1) for x in up_ms], "download_ms": [round(x, 1) for x in down_ms],
                       "d2h_copy_gbps": round(d2h, 1)}
        del Hh, Sh

    # accuracy of the timed build (after the timed region): whole columns vs the oracle
    ref = None
    if rank == 0 and not args.no_error and st.get("s_form") != hsgen.S_LEGENDRE and args.l_nonsph < 0:
        cols = error_columns(n)
        ci = torch.tensor(cols, device=dev)
        Hc, Sc = H.mT[:, ci].cpu().numpy(), S.mT[:, ci].cpu().numpy()
        ref = oracle_columns(sysm, kv_host, cols)
        line["error"] = dict(column_errors(Hc, Sc, ref), tolerance=1e-11 if precision == hsgen.SPLIT else 1e-12,
                             sample=f"{len(cols)} whole columns {cols} (all rows of the upper triangle) vs the "
                                    f"oracle ({ref['seconds']:.0f} s on the host cores)")
    g.close()

    if rank == 0 and precision == hsgen.SPLIT and not args.no_fp64_compare:
        # the plain form on the same workload: one timed FP64 build (after a
        # small build that loads its kernels), with its own error
        g64 = hsgen.Generator(sysm, device=local, precision=hsgen.FP64, s_form=s_form)
        g64.build(kv[:64])
        H.zero_()
        S.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk64:
            e0.record(stream)
            g64.build(kv, H, S)
            e1.record(stream)
            torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1) * 1e-3
        st64 = g64.stats()
        f64 = {"s_per_kpoint": t64, "eff_tflops": fal["total"] / t64 / 1e12, "steps": 1, "warmup": 0,
               "phases_ms": {k: st64[k] for k in ("ms_coefficients", "ms_tapply", "ms_contract", "ms_total")},
               "roofline": roofline(st64, f_contract, st64["ms_contract"], hsgen.FP64, peaks, clk64.summary(),
                                    args, hsgen),
               "split_speedup": t64 / s_per_k}
        if ref is not None:
            ci = torch.tensor(ref["cols"], device=dev)
            Hc, Sc = H.mT[:, ci].cpu().numpy(), S.mT[:, ci].cpu().numpy()
            f64["error"] = dict(column_errors(Hc, Sc, ref), tolerance=1e-12)
        line["fp64_form"] = f64
        g64.close()

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle

        full, spent, model = oracle_sample_time(sysm, kv_host, args.ref_columns)
        line["cpu_baseline"] = {"value": full, "unit": "s/k-point", "cores": oracle.threads(), "kind": "oracle",
                                "sample": f"{args.ref_columns} columns + {args.ref_columns ** 2} entries "
                                          f"({spent:.1f} s of CPU work), extrapolated to the full k-point"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
