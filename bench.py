#!/usr/bin/env python3
"""Dash update throughput on GB300: rows absorbed per second and p50/p99
update latency, mixed precision vs FP64, on a synthetic planted stream.

    python bench.py [--gpus N --steps K --warmup W] [--workload c4] [--impl reference]

One step = one dash_update (Algorithm 1) over one batch of new rows that is
already resident in HBM.  N > 1 (torchrun) runs N independent replicas, one
stream per GPU (the path has no exchange in this build), and reports the
whole-job rows/s over the slowest rank.  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Dash update rows/s & p50/p99 latency, mixed-prec vs FP64 on 1 GB300"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
def fp64_peak_tflops():
    """FP64 peak of this device in TFLOP/s (2 flops per FMA), measured live by
    the library's FMA-chain kernel (dash_measure_fp64_fma)."""
    from paper_2305_18376_gb300._native import measure_fp64_fma
    return 2.0 * measure_fp64_fma() / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c4")
    ap.add_argument("--precision", default="f16x3", choices=["fp32", "f16x3"])
    ap.add_argument("--row-path", default="auto", choices=["auto", "fused", "split", "split-warp"],
                    help="mode-P row pipeline (f16x3 only)")
    ap.add_argument("--init-iters", type=int, default=3)
    ap.add_argument("--graph", action="store_true",
                    help="submit each update as one CUDA graph (no per-kernel profile then)")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-slices", type=int, default=50,
                    help="slices in the oracle's bounded CPU sample")
    ap.add_argument("--profile-out", default="", help="write the per-kernel profile here")
    ap.add_argument("--init-max-rows", type=int, default=0,
                    help="clip the initial slices' row counts (reduced cases for profiling only)")
    ap.add_argument("--k0", type=int, default=0, help="override the initial slice count "
                    "(reduced cases for profiling only; the bench line uses the workload's)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--q-steps", type=int, default=4,
                    help="timed updates of the constrained-mode (Q) measurement; 0 skips it")
    ap.add_argument("--q-init-iters", type=int, default=2)
    ap.add_argument("--cycle-scan", action="store_true",
                    help="update time against update size for the dual-way, rows-only and "
                    "slices-only streaming settings (prints one JSON line; not the bench line)")
    ap.add_argument("--lambda-sweep", action="store_true",
                    help="local and global errors of a drifting stream for several forgetting "
                    "factors (prints one JSON line; not the bench line)")
    ap.add_argument("--serving", action="store_true",
                    help="the serving loop on many independent streams with Poisson arrivals: "
                    "p50/p99 update latency and rows/s, mixed and FP64 (prints one JSON line; "
                    "not the bench line)")
    ap.add_argument("--serve-streams", type=int, default=8)
    ap.add_argument("--serve-seconds", type=float, default=0.5)
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-k0-max", type=int, default=1000)
    ap.add_argument("--serve-budget-gb", type=float, default=64.0)
    ap.add_argument("--serve-profile", action="store_true",
                    help="per-kernel profile of every serving model (adds events and host work)")
    ap.add_argument("--serve-precisions", default="f16x3,fp64")
    ap.add_argument("--serve-init-iters", type=int, default=10,
                    help="static ALS iterations of each stream's initial fit (untimed); Algorithm 1 "
                         "does not fix the scale of S_k against V, and a poorly fitted start drifts")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


# ---------------------------------------------------------------------------
# nvidia-smi clock sampling during the timed region
# ---------------------------------------------------------------------------
CLOCK_Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.idx = gpu_index
        self.proc = None

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx),
                                          f"--query-gpu={CLOCK_Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        mhz, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                mhz.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not mhz:
            return None
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(mhz)}


# ---------------------------------------------------------------------------
# algorithmic work: the bytes (or flops) each kernel must move per launch
# ---------------------------------------------------------------------------
def algorithmic(kernel: str, plan: dict, N: int, K_all: int, J: int, R: int, tsize: int,
                isize: int):
    """(bytes, flops) one launch must move / do, by kernel.  plan: the
    library's account of the batch (dash_last_plan), averaged over the timed
    updates: rows and slices of the fused tiles, chunked-path rows, rows of
    the general kernels.  Per-slice mode-P state is c_k (R), the symmetric
    D_k (R(R+1)/2) and W(k,:) (R), FP64-sized, read and written."""
    per_slice = (R + R * (R + 1) // 2 + R) * 8 * 2
    tr, ts = plan.get("tile_rows", 0), plan.get("tile_slices", 0)
    cr, gr = plan.get("chunk_rows", 0), plan.get("general_rows", 0)
    if kernel == "k_rows_fused":         # one read of every tile row, U written
        return tr * J * isize + tr * R * 4 + ts * per_slice, 4 * tr * J * R
    if kernel in ("k_xq_tc", "k_xq_umma"):   # X read, P' (mode Q: P) written
        n = cr + gr
        return n * J * isize + n * R * 4, 2 * n * J * R
    if kernel == "k_q_arows":            # P and A rows, R values each (W rows from L2)
        return 2 * N * R * tsize, 2 * N * R * R
    if kernel == "k_f_tc":               # X read, Ũ fragment blocks (16 rows each) read
        nt = -(-R // 8)
        return cr * J * isize + -(-cr // 16) * (512 * nt + 16), 2 * cr * J * R
    if kernel == "k_f_umma":             # X read, U rows read (Ũ = U ∘ w built in the kernel)
        return cr * J * isize + cr * R * 4, 2 * cr * J * R
    if kernel == "k_utilde":             # U read, U ∘ w written (rank padded to 8)
        return cr * R * 4 + cr * (-(-R // 8) * 8) * 4, cr * R
    if kernel == "k_xv":
        n = cr + gr
        return n * J * isize + n * R * tsize, 2 * n * J * R
    if kernel == "k_f":
        n = cr + gr
        return n * J * isize + n * R * tsize, 2 * n * J * R
    if kernel == "k_big_b":              # P' read, U written
        return 2 * cr * R * 4, 2 * cr * R * R
    if kernel == "k_big_c":              # state of every slice not finished in a tile
        return (K_all - ts) * per_slice, 0
    if kernel == "k_slices":
        return 2 * N * R * tsize + K_all * per_slice, N * (3 * R * R) + K_all * (R ** 3 // 3)
    # mode Q (all rows general); Y_k is K×R×J in the product type
    Yb = K_all * R * J * tsize
    if kernel == "k_q_y":                # Y read + written, X read, new Q rows read
        return 2 * Yb + N * J * isize + N * R * tsize, 2 * K_all * R * J * R + 2 * N * R * J
    if kernel in ("k_q_vpart", "k_q_w"):  # one pass over Y
        return Yb, 2 * K_all * R * J * R
    if kernel == "k_q_out":              # X read, Q rows read
        return N * J * isize + N * R * tsize, 2 * N * J * R
    if kernel == "k_q_lt":               # L, E, B^1/2 read + written, carry written, A read, Q written
        return K_all * R * R * 8 * 7 + 2 * N * R * tsize, 0
    return None, None


def step_bytes(N, K_all, J, R, isize):
    """§8(d) algorithmic bytes of one mode-P update: X read once, U written,
    the per-slice helpers read and written."""
    return N * J * isize + N * R * 4 + K_all * (R + R * (R + 1) // 2 + R) * 8 * 2


def step_bytes_q(N, K_all, J, R, isize, tsize=4):
    """Algorithmic bytes of one mode-Q update: X read once, the new Q rows
    written, Y_k read and written once (its update, fused with the H-MTTKRP)
    and read twice more (the V-MTTKRP needs the new H, the W step the new V),
    the per-slice factors L_k, E_k, B_k^{1/2} read and written."""
    return (N * J * isize + N * R * tsize + 4 * K_all * R * J * tsize
            + K_all * R * R * 8 * 6)


def src_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2305_18376_gb300", "csrc")
    for fn in sorted(os.listdir(d)):
        h.update(open(os.path.join(d, fn), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if the
    kernel's sources are unchanged since the capture (else None)."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(kernel)
    if not e:
        return None
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2305_18376_gb300", "csrc")
    for fn in e.get("src_files", []):
        h.update(open(os.path.join(csrc, fn), "rb").read())
    if h.hexdigest()[:16] != e.get("src_sha"):
        return None
    return e.get("dram_bytes_per_launch_full")


# ---------------------------------------------------------------------------
# CPU baseline / reference arm: the FP64 oracle on a bounded sample
# ---------------------------------------------------------------------------
def oracle_sample(wname: str, n_slices: int, n_updates: int, warm: int = 0, init_iters: int = 3):
    """Time the FP64 oracle's mode-P update (Algorithm 1) on a bounded sample
    of workload `wname`: the same stream recipe with n_slices initial slices
    (new slices per update scaled down in proportion).

    The starting state is fitted the way the GPU arm fits its own: the
    workload's initial row recipe, then `init_iters` static ALS iterations
    from V0 ~ U(0,1), W0 = 1, each one oracle update on empty helpers (λ = 0,
    which equals one static ALS iteration), then the helpers of the final
    factors (Eqs. 6-9).  Algorithm 1 fixes no scale between S_k and V, so from
    an unfitted start (one iteration, or slices of a few rows) W grows and V
    shrinks without bound within a few updates; a fitted start stays put."""
    import numpy as np
    import torch
    from oracle import dash_oracle as O
    from synth.planted import PlantedStream, workload
    try:
        from threadpoolctl import threadpool_info
        blas = max([i.get("num_threads", 1) for i in threadpool_info()] or [1])
    except Exception:
        blas = os.cpu_count() or 1
    w = workload(wname)
    w = type(w)(**{**w.__dict__, "K0": n_slices, "steps": warm + n_updates,
                   "new_slices_per_step": max(1, w.new_slices_per_step * n_slices // w.K0)})
    s = PlantedStream(w, dtype=torch.float32)
    b0 = s.batch(0)
    segs0 = [(k, x.double().numpy()) for k, x in b0.segments()]
    t_init = time.perf_counter()
    st = O.empty_state_p(np.random.default_rng(0).random((w.J, w.R)))
    U = {}
    for it in range(init_iters):
        st, U = O.dash_update_p(st, segs0, b0.n_new if it == 0 else 0, 0.0)
    st = O.init_helpers_p([x for _, x in segs0], [U[k] for k in range(len(segs0))], st.W, st.V)
    t_init = time.perf_counter() - t_init
    times, rows = [], []
    for t in range(1, warm + n_updates + 1):
        b = s.batch(t)
        segs = [(k, x.double().numpy()) for k, x in b.segments()]
        t0 = time.perf_counter()
        st, _ = O.dash_update_p(st, segs, b.n_new, w.lam)
        dt = time.perf_counter() - t0
        if t > warm:
            times.append(dt)
            rows.append(b.n_rows)
    if not all(np.isfinite(st.V).ravel()) or not all(np.isfinite(st.W).ravel()):
        raise RuntimeError("oracle sample state went non-finite")
    return {"rows": rows, "times": times, "cores": blas, "nproc": os.cpu_count(),
            "init_s": t_init, "max_abs_W": float(np.abs(st.W).max()),
            "sample": f"{wname} update recipe on K0={n_slices} slices (J={w.J}, R={w.R}, the "
                      f"workload's initial row recipe, {b0.n_rows} rows, fitted by "
                      f"{init_iters} untimed static ALS iterations), {n_updates} timed "
                      f"updates after {warm} untimed, oracle mode P in numpy float64"}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from synth.planted import workload
    w = workload(a.workload)
    r = oracle_sample(a.workload, a.cpu_slices, a.steps, warm=a.warmup,
                      init_iters=a.init_iters)
    tot_rows, tot_t = sum(r["rows"]), sum(r["times"])
    v = tot_rows / tot_t
    lat = sorted(r["times"])
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "rows/s", "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * tot_t / len(r["times"]),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(w, a),
        "latency": {"p50_ms": 1e3 * statistics.median(lat), "p99_ms": 1e3 * lat[-1]},
        "cpu_baseline": {"value": v, "unit": "rows/s", "cores": r["cores"], "kind": "oracle",
                         "sample": r["sample"], "nproc": r["nproc"]},
        "e2e": {"value": v, "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(w, a):
    return {"workload": f"{w.name}: planted PARAFAC2 stream, K0={w.K0}, J={w.J}, R={w.R}, "
                        f"init rows {w.init_rows}, +{w.rows_per_step} rows per slice and "
                        f"+{w.new_slices_per_step} slices {w.new_slice_rows} per update, "
                        f"sigma={w.sigma}, lambda={w.lam}",
            "mode": "P (Algorithm 1)", "precision": a.precision, "row_path": a.row_path,
            "input": "f32",
            "init": f"{a.init_iters} static ALS iterations on the GPU",
            "l2": "inputs larger than L2 (each step's X_new is GBs)"}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(a):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2305_18376_gb300 import DashModel
    from synth.planted import PlantedStream, workload

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()

    w = workload(a.workload)
    if a.k0:
        w = type(w)(**{**w.__dict__, "K0": a.k0})
    if a.init_max_rows:
        ir = tuple(w.init_rows)
        w = type(w)(**{**w.__dict__, "init_rows": ir[:-1] + (min(ir[-1], a.init_max_rows),)})
    n_batches = a.warmup + a.steps
    if n_batches > w.steps:
        w = type(w)(**{**w.__dict__, "steps": n_batches})
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    s = PlantedStream(w, device="cuda", dtype=torch.float32, seed=w.seed + 1000 * rank)
    b0 = s.batch(0)
    batches = [s.batch(t) for t in range(1, n_batches + 1)]
    del s
    max_rows = max([b0.n_rows] + [b.n_rows for b in batches])
    max_seg = max([b0.slice_ids.numel()] + [b.slice_ids.numel() for b in batches])
    K_total = w.K0 + w.new_slices_per_step * n_batches
    step_rows = max(b.n_rows for b in batches)
    m = DashModel(w.J, w.R, w.lam, precision=a.precision, input_dtype="f32",
                  max_slices=K_total + 8, max_rows=max_rows, max_segments=max_seg + 8,
                  stream=stream.cuda_stream, max_staged_rows=step_rows)
    m.set_row_path(a.row_path)
    if a.graph:
        m.set_graph(True)
    V0 = np.random.default_rng(7).random((w.J, w.R))
    m.set_factors(V0)
    t0 = time.perf_counter()
    m.fit_initial_device(b0.slice_ids.numpy(), b0.row_ptr.numpy(), b0.X, a.init_iters)
    m.sync()
    init_s = time.perf_counter() - t0
    fit_init = m.fitness()[0]
    # the constrained mode is fitted on the same initial tensor now, measured later
    mq = None
    if a.q_steps > 0 and world == 1:
        mq = DashModel(w.J, w.R, w.lam, mode="Q", precision=a.precision, input_dtype="f32",
                       max_slices=K_total + 8, max_rows=max_rows, max_segments=max_seg + 8,
                       stream=stream.cuda_stream, max_staged_rows=1)
        mq.set_factors(V0)
        t1 = time.perf_counter()
        mq.fit_initial_device(b0.slice_ids.numpy(), b0.row_ptr.numpy(), b0.X, a.q_init_iters)
        mq.sync()
        q_init_s = time.perf_counter() - t1
    del b0
    torch.cuda.empty_cache()
    # the last warm-up update runs with the in-kernel phase clocks (extra
    # work inside the kernels), so the timed updates carry only the events
    phase_rep = {}
    for i, b in enumerate(batches[: a.warmup]):
        if i == a.warmup - 1 and not a.graph:
            m.profile(True, phases=True)
        m.update_device(b.slice_ids.numpy(), b.row_ptr.numpy(), b.X)
    m.sync()
    if a.warmup > 0 and not a.graph:
        phase_rep = {k: v for k, v in m.profile_report().items() if "." in k and not k.startswith("host.")}
        m.profile(False)
    snap = m.get_state_p() if (rank == 0 and not a.no_fp64) else None
    timed = batches[a.warmup:]
    # ---- timed region (device-resident inputs) ----------------------------
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in timed]
    m.profile(not a.graph)
    l0 = m.launch_count()
    fits = []
    sampler = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e_start.record(stream)
    plans = []
    torch.cuda.nvtx.range_push("dash_p_timed")    # ncu --nvtx-include dash_p_timed/
    for (ea, eb), b in zip(evs, timed):
        ea.record(stream)
        m.update_device(b.slice_ids.numpy(), b.row_ptr.numpy(), b.X)
        eb.record(stream)
        plans.append(m.last_plan())
    e_end.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    launches = m.launch_count() - l0
    timeouts, fallbacks = m.counters()
    tune = m.autotune_result()
    prof = m.profile_report()
    m.profile(False)
    elapsed = e_start.elapsed_time(e_end) / 1e3
    lat = sorted(ea.elapsed_time(eb) for ea, eb in evs)
    rows = sum(b.n_rows for b in timed)
    t_max = elapsed
    if world > 1:
        tt = torch.tensor([elapsed], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max = float(tt.item())
        rr = torch.tensor([float(rows)], device="cuda")
        dist.all_reduce(rr)
        rows_all = float(rr.item())
    else:
        rows_all = float(rows)
    value = rows_all / t_max
    fit_last = m.fitness()[0]
    # ---- FP64 path on the same state and inputs (rank 0) -------------------
    fp64 = None
    if snap is not None:
        m64 = DashModel(w.J, w.R, w.lam, precision="fp64", input_dtype="f32",
                        max_slices=K_total + 8, max_rows=step_rows, max_segments=max_seg + 8,
                        stream=stream.cuda_stream, max_staged_rows=1)
        m64.set_state_p(**snap)
        m_fit, d_fit = [], []
        # replay the mixed model from the same snapshot for a per-step fitness diff
        mm = DashModel(w.J, w.R, w.lam, precision=a.precision, input_dtype="f32",
                       max_slices=K_total + 8, max_rows=step_rows, max_segments=max_seg + 8,
                       stream=stream.cuda_stream, max_staged_rows=1)
        mm.set_state_p(**snap)
        mm.set_row_path(a.row_path)
        ev64 = []
        for b in timed:
            ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ea.record(stream)
            m64.update_device(b.slice_ids.numpy(), b.row_ptr.numpy(), b.X)
            eb.record(stream)
            ev64.append((ea, eb))
            f64v = m64.fitness()[0]
            mm.update_device(b.slice_ids.numpy(), b.row_ptr.numpy(), b.X)
            fmv = mm.fitness()[0]
            m_fit.append(f64v)
            d_fit.append(abs(fmv - f64v))
        torch.cuda.synchronize()
        l64 = sorted(ea.elapsed_time(eb) for ea, eb in ev64)
        st64, stm = m64.get_state_p(), mm.get_state_p()
        err = {k: float(np.max(np.abs(stm[k] - st64[k])) / max(np.max(np.abs(st64[k])), 1e-300))
               for k in ("V", "W", "c", "D", "F", "G")}
        p64 = fp64_peak_tflops()
        fl64 = 4.0 * w.J * w.R * rows / len(timed)          # X·V and Xᵀ(U S) per update
        fp64 = {"value": rows / (sum(l64) / 1e3), "unit": "rows/s",
                "roofline": {"bound": "alu", "achieved": fl64 / (sum(l64) / len(l64) / 1e3) / 1e12,
                             "peak": p64, "unit": "TFLOP/s",
                             "frac": fl64 / (sum(l64) / len(l64) / 1e3) / 1e12 / p64,
                             "peak_source": "measured live: dash_measure_fp64_fma (FMA chains, 2 flops per FMA)",
                             "work": "4·J·R flops per row (both bulk products)"},
                "ms_per_step": sum(l64) / len(l64), "p50_ms": statistics.median(l64),
                "p99_ms": l64[-1], "fitness_mean": float(np.mean(m_fit)),
                "max_abs_fitness_diff_mixed_vs_fp64": float(max(d_fit)),
                "max_rel_err_mixed_vs_fp64": err}
        m64.close()
        mm.close()
    # ---- end to end through the C ABI with host buffers --------------------
    e2e = None
    if not a.no_e2e:
        hosts = []
        for b in timed[: min(2, len(timed))]:
            hx = torch.empty(b.X.shape, dtype=b.X.dtype, pin_memory=True)
            hx.copy_(b.X)
            hosts.append((b, hx))
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        h2d = d2h = 0
        erows = 0
        b, hx = hosts[0]
        m.append_batch(b.slice_ids.numpy(), b.row_ptr.numpy(), hx)
        step_s = []
        for i in range(len(timed)):
            b, hx = hosts[i % len(hosts)]
            ts0 = time.perf_counter()
            m.update()
            if i + 1 < len(timed):                # the next step's copy overlaps this update
                nb, nhx = hosts[(i + 1) % len(hosts)]
                m.append_batch(nb.slice_ids.numpy(), nb.row_ptr.numpy(), nhx)
            m.fitness()                           # D2H read of the step's result
            step_s.append(time.perf_counter() - ts0)
            h2d += hx.numel() * hx.element_size() + 16 * b.slice_ids.numel()
            d2h += 24
            erows += b.n_rows
        torch.cuda.synchronize()
        et = time.perf_counter() - t0
        if world > 1:
            tt = torch.tensor([et], device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            et = float(tt.item())
        e2e = {"value": erows * world / et, "unit": "rows/s",
               "h2d_bytes_per_step": h2d // len(timed), "d2h_bytes_per_step": d2h // len(timed),
               # host time per step (each step waits for its own copy): the
               # median is the steady state, the maximum shows slow copies
               "step_ms_p50": statistics.median(step_s) * 1e3, "step_ms_max": max(step_s) * 1e3,
               "h2d_gbs_at_p50": h2d / len(timed) / statistics.median(step_s) / 1e9}
    # ---- roofline of the dominant kernel ------------------------------------
    pk, pk_kind = peaks()
    Nm = int(statistics.mean(b.n_rows for b in timed))
    K_all = w.K0 + w.new_slices_per_step * (a.warmup + len(timed))
    # the dominant kernel: by time, among launched kernels (not the in-kernel
    # phase counters "kernel.phase" nor the host timers "host.*")
    prof = {k: v for k, v in prof.items() if "." not in k or k.startswith("host.")}
    prof.update(phase_rep)           # phase clocks: one (warm-up) update
    launched = {k: v for k, v in prof.items() if "." not in k}
    top = max(launched.items(), key=lambda kv: kv[1][1]) if launched else None
    roof = None
    kernels = {}
    plan = {k: statistics.mean(p[k] for p in plans) for k in plans[0]}
    for name, (n, ms) in prof.items():
        by, fl = algorithmic(name, plan, Nm, K_all, w.J, w.R, 4, 4)
        d = {"launches": n, "ms_total": ms, "ms_per_launch": ms / n}
        if by:
            d["gbs"] = by / (ms / n / 1e3) / 1e9
            d["gflops"] = fl / (ms / n / 1e3) / 1e9
        kernels[name] = d
    if top:
        name, (n, ms) = top
        by, fl = algorithmic(name, plan, Nm, K_all, w.J, w.R, 4, 4)
        if by:
            per = ms / n / 1e3
            ach = by / per / 1e9
            hbm = pk["hbm_gbs"]
            if name == "k_slices":
                p64 = fp64_peak_tflops()
                roof = {"bound": "alu", "achieved": fl / per / 1e12, "peak": p64,
                        "unit": "TFLOP/s", "frac": fl / per / 1e12 / p64,
                        "traffic": ncu_traffic(name), "kernel": name,
                        "peak_source": "measured live: dash_measure_fp64_fma (FMA chains, 2 flops per FMA)"}
            else:
                roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                        "frac": ach / hbm, "traffic": ncu_traffic(name), "kernel": name,
                        "peak_source": f"{pk_kind} (MEASURED_PEAKS.json hbm_gbs)"}
    sb = step_bytes(Nm, K_all, w.J, w.R, 4)
    mode_q = None
    if mq is not None:
        mode_q = measure_mode_q(a, w, mq, batches, stream, K_total, step_rows, max_seg, pk, q_init_s)
        mq.close()
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        r = oracle_sample(a.workload, a.cpu_slices, 12, init_iters=a.init_iters)
        cpu = {"value": sum(r["rows"]) / sum(r["times"]), "unit": "rows/s", "cores": r["cores"],
               "kind": "oracle", "sample": r["sample"], "nproc": r["nproc"]}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * t_max / len(timed),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if a.precision == "fp32" else "f16x3",
            "data": "synthetic", "config": workload_config(w, a),
            "latency": {"p50_ms": statistics.median(lat), "p99_ms": lat[-1]},
            "rows_per_step": Nm, "slices": K_all, "plan": plan,
            "fitness": {"init": fit_init, "last_step": fit_last},
            "fp64": fp64, "e2e": e2e, "gpu_launches": launches,
            "roofline": roof,
            "step_roofline": {"bound": "hbm", "algorithmic_bytes": sb,
                              "achieved": sb / (t_max / len(timed)) / 1e9, "peak": pk["hbm_gbs"],
                              "unit": "GB/s", "frac": sb / (t_max / len(timed)) / 1e9 / pk["hbm_gbs"]},
            "kernels": kernels, "mode_q": mode_q, "cpu_baseline": cpu, "clocks": clocks,
            "init_seconds": init_s, "src_sha": src_hash(),
            "diagnostics": {"wait_timeouts": timeouts, "fp64_fallback_solves": fallbacks},
            "xq_autotune": tune,
        }
        print(json.dumps(line), flush=True)
        if a.profile_out:
            json.dump({"kernels": kernels, "config": line["config"]}, open(a.profile_out, "w"),
                      indent=1)
    m.close()
    if world > 1:
        dist.destroy_process_group()


def measure_mode_q(a, w, mq, batches, stream, K_total, step_rows, max_seg, pk, init_s):
    """The constrained mode (U_k = Q_k H S_k) on the same stream: one untimed
    update, then q_steps timed ones (CUDA events on the model's stream), the
    FP64 path replayed from a snapshot for two of them."""
    import numpy as np
    import torch
    from paper_2305_18376_gb300 import DashModel
    n_t = min(a.q_steps, len(batches) - 1)
    mq.update_device(batches[0].slice_ids.numpy(), batches[0].row_ptr.numpy(), batches[0].X)
    mq.sync()
    snap = None if a.no_fp64 else mq.get_state_q()
    timed = batches[1:1 + n_t]
    mq.profile(True, phases=True)   # k_q_lt's phase clocks: a few clock reads per slice
    evs = []
    torch.cuda.nvtx.range_push("dash_q_timed")    # ncu --nvtx-include dash_q_timed/
    for b in timed:
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea.record(stream)
        mq.update_device(b.slice_ids.numpy(), b.row_ptr.numpy(), b.X)
        eb.record(stream)
        evs.append((ea, eb))
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    prof = mq.profile_report()
    mq.profile(False)
    lat = sorted(ea.elapsed_time(eb) for ea, eb in evs)
    rows = sum(b.n_rows for b in timed)
    Nm = int(statistics.mean(b.n_rows for b in timed))
    K_all = w.K0 + w.new_slices_per_step * (1 + n_t)
    kernels = {}
    for name, (n, ms) in prof.items():
        by, fl = algorithmic(name, {"general_rows": Nm}, Nm, K_all, w.J, w.R, 4, 4)
        d = {"launches": n, "ms_total": ms, "ms_per_launch": ms / n}
        if by:
            d["gbs"] = by / (ms / n / 1e3) / 1e9
        kernels[name] = d
    sbq = step_bytes_q(Nm, K_all, w.J, w.R, 4)
    t_step = sum(lat) / len(lat) / 1e3
    out = {"value": rows / (sum(lat) / 1e3), "unit": "rows/s", "steps": n_t, "warmup": 1,
           "ms_per_step": 1e3 * t_step, "p50_ms": statistics.median(lat), "p99_ms": lat[-1],
           "init_seconds": init_s, "init_iters": a.q_init_iters, "fitness": mq.fitness()[0],
           "step_roofline": {"bound": "hbm", "algorithmic_bytes": sbq, "achieved": sbq / t_step / 1e9,
                             "peak": pk["hbm_gbs"], "unit": "GB/s",
                             "frac": sbq / t_step / 1e9 / pk["hbm_gbs"]},
           "kernels": kernels}
    if snap is not None:
        n64 = min(2, n_t)
        m64 = DashModel(w.J, w.R, w.lam, mode="Q", precision="fp64", input_dtype="f32",
                        max_slices=K_total + 8, max_rows=step_rows, max_segments=max_seg + 8,
                        stream=stream.cuda_stream, max_staged_rows=1)
        m64.set_state_q(**snap)
        mm = DashModel(w.J, w.R, w.lam, mode="Q", precision=a.precision, input_dtype="f32",
                       max_slices=K_total + 8, max_rows=step_rows, max_segments=max_seg + 8,
                       stream=stream.cuda_stream, max_staged_rows=1)
        mm.set_state_q(**snap)
        del snap
        l64, dfit = [], []
        for b in timed[:n64]:
            ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ea.record(stream)
            m64.update_device(b.slice_ids.numpy(), b.row_ptr.numpy(), b.X)
            eb.record(stream)
            f64v = m64.fitness()[0]
            mm.update_device(b.slice_ids.numpy(), b.row_ptr.numpy(), b.X)
            dfit.append(abs(mm.fitness()[0] - f64v))
            torch.cuda.synchronize()
            l64.append(ea.elapsed_time(eb))
        s64, smx = m64.get_state_q(), mm.get_state_q()
        err = {k: float(np.max(np.abs(smx[k] - s64[k])) / max(np.max(np.abs(s64[k])), 1e-300))
               for k in ("V", "H", "W", "L", "Y")}
        out["fp64"] = {"value": sum(b.n_rows for b in timed[:n64]) / (sum(l64) / 1e3),
                       "unit": "rows/s", "ms_per_step": sum(l64) / len(l64), "steps": n64,
                       "max_abs_fitness_diff_mixed_vs_fp64": float(max(dfit)),
                       "max_rel_err_mixed_vs_fp64": err}
        m64.close()
        mm.close()
    return out


# ---------------------------------------------------------------------------
# Extra workloads: update-cycle scan (the paper's settings 2-4 and Fig. 5's
# linearity) and the forgetting-factor sweep (§4.4)
# ---------------------------------------------------------------------------
def derive_batch(b, K_cur, scale, rows=True, slices=True):
    """A batch derived from planted batch b: each segment keeps its first
    ceil(scale·n) rows; rows=False drops the segments of existing slices,
    slices=False drops the new slices (new slices are renumbered from K_cur).
    Returns (slice_ids, row_ptr, X) with X on b.X's device."""
    import math
    import torch
    ids, rp = b.slice_ids.tolist(), b.row_ptr.tolist()
    keep_ids, take, nxt = [], [], K_cur
    for q, k in enumerate(ids):
        n = rp[q + 1] - rp[q]
        is_new = k >= b.K_before
        if (is_new and not slices) or (not is_new and (not rows or k >= K_cur)):
            continue
        m = min(n, max(1 if is_new else 0, math.ceil(scale * n)))
        if is_new:
            keep_ids.append(nxt)
            nxt += 1
        else:
            keep_ids.append(k)
        take.append((rp[q], m))
    import numpy as np
    starts = np.array([r0 for r0, _ in take], dtype=np.int64)
    counts = np.array([m for _, m in take], dtype=np.int64)
    row_ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    idx = np.repeat(starts - row_ptr[:-1], counts) + np.arange(int(row_ptr[-1]), dtype=np.int64)
    X = b.X.index_select(0, torch.from_numpy(idx).to(b.X.device)).contiguous()
    return keep_ids, row_ptr.tolist(), X, nxt - K_cur


def run_cycle_scan(a):
    import numpy as np
    import torch

    from paper_2305_18376_gb300 import DashModel
    from synth.planted import PlantedStream, workload

    w = workload(a.workload)
    if a.k0:
        w = type(w)(**{**w.__dict__, "K0": a.k0})
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    s = PlantedStream(w, device="cuda", dtype=torch.float32, seed=w.seed + 1000)
    b0 = s.batch(0)
    batches = [s.batch(t) for t in range(1, 6)]
    max_rows = max([b0.n_rows] + [b.n_rows for b in batches])
    max_seg = max(b.slice_ids.numel() for b in [b0] + batches) + 8
    K_total = w.K0 + 5 * w.new_slices_per_step + 8

    def model():
        return DashModel(w.J, w.R, w.lam, precision=a.precision, input_dtype="f32",
                         max_slices=K_total, max_rows=max_rows, max_segments=max_seg,
                         stream=stream.cuda_stream, max_staged_rows=1)
    m = model()
    m.set_row_path(a.row_path)
    m.set_factors(np.random.default_rng(7).random((w.J, w.R)))
    m.fit_initial_device(b0.slice_ids.numpy(), b0.row_ptr.numpy(), b0.X, a.init_iters)
    m.sync()
    snap, K_snap = m.get_state_p(), m.K
    m.close()
    del b0
    out = {}
    for variant, rows, slices in (("dual-way", True, True), ("rows-only", True, False),
                                  ("slices-only", False, True)):
        pts = []
        for scale in (0.2, 0.4, 0.6, 0.8, 1.0):
            mm = model()
            mm.set_row_path(a.row_path)
            mm.set_state_p(**snap)
            K, times, nrows = K_snap, [], []
            for t, b in enumerate(batches):
                ids, rp, X, n_new = derive_batch(b, K, scale, rows, slices)
                ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ea.record(stream)
                mm.update_device(np.asarray(ids), np.asarray(rp), X)
                eb.record(stream)
                K += n_new
                if t >= 1:                 # the first update is a warm-up
                    times.append((ea, eb))
                    nrows.append(rp[-1])
            torch.cuda.synchronize()
            ms = [ea.elapsed_time(eb) for ea, eb in times]
            pts.append({"scale": scale, "rows_per_update": float(np.mean(nrows)),
                        "ms_per_update": float(np.median(ms))})
            mm.close()
        x = np.array([p["rows_per_update"] for p in pts])
        y = np.array([p["ms_per_update"] for p in pts])
        slope, icpt = np.polyfit(x, y, 1)
        r2 = 1.0 - float(np.sum((y - (slope * x + icpt)) ** 2) / max(np.sum((y - y.mean()) ** 2), 1e-30))
        out[variant] = {"points": pts, "linear_fit": {"ms_per_million_rows": float(slope * 1e6),
                                                      "intercept_ms": float(icpt), "r2": r2}}
    print(json.dumps({"metric": "update time vs update size (update cycle scan)",
                      "workload": workload_config(w, a)["workload"],
                      "row_path": a.row_path, "precision": a.precision, "settings": out}))


def run_lambda_sweep(a):
    import numpy as np
    import torch

    from paper_2305_18376_gb300 import DashModel
    from synth.planted import PlantedStream, workload

    w = workload("c2", K0=300, init_rows=("uniform", 50, 300), new_slice_rows=("uniform", 50, 100),
                 steps=20, drift=0.02)
    lams = (0.1, 0.3, 0.5, 0.7, 0.9)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    res = {}
    for lam in lams:
        s = PlantedStream(w, device="cuda", dtype=torch.float32, seed=w.seed + 1000)
        bs = [s.batch(t) for t in range(w.steps + 1)]
        m = DashModel(w.J, w.R, lam, precision=a.precision, input_dtype="f32",
                      max_slices=w.K0 + w.new_slices_per_step * w.steps + 8,
                      max_rows=max(b.n_rows for b in bs), max_segments=4096,
                      stream=stream.cuda_stream, max_staged_rows=1)
        m.set_factors(np.random.default_rng(7).random((w.J, w.R)))
        m.fit_initial_device(bs[0].slice_ids.numpy(), bs[0].row_ptr.numpy(), bs[0].X, a.init_iters)
        ids_all, rp_all, X_all, U_all = [], [0], [], []

        def add(b, U):
            rp = b.row_ptr.tolist()
            for q, k in enumerate(b.slice_ids.tolist()):
                ids_all.append(k)
                rp_all.append(rp_all[-1] + rp[q + 1] - rp[q])
            X_all.append(b.X)
            U_all.append(torch.from_numpy(U))
        add(bs[0], m.new_rows())
        loc, glo = [], []
        for t in range(1, w.steps + 1):
            b = bs[t]
            m.update_device(b.slice_ids.numpy(), b.row_ptr.numpy(), b.X)
            _, fd, _ = m.local_errors()
            loc.append((1.0 - fd) ** 2)            # Σ||X_new − X̂||² / Σ||X_new||²
            add(b, m.new_rows())
            e2, x2, _ = m.rows_error(ids_all, rp_all, torch.cat(X_all), torch.cat(U_all).cuda())
            glo.append(e2 / x2)
        res[str(lam)] = {"local_error_mean": float(np.mean(loc)), "global_error_mean": float(np.mean(glo)),
                         "local_error_last": loc[-1], "global_error_last": glo[-1]}
        m.close()
    print(json.dumps({"metric": "forgetting-factor sweep: mean local and global relative squared error",
                      "workload": (f"c2-shaped drifting stream: K0={w.K0}, J={w.J}, R={w.R}, "
                                   f"{w.steps} updates, +1 row per slice and +{w.new_slices_per_step} "
                                   f"slices per update, drift {w.drift}, sigma {w.sigma}"),
                      "precision": a.precision, "lambda": res}))


def _replay_requests(load, s, b0, pool, K0, tdt, Request, init_iters):
    """Stream s's requests: its initial fit, then one update per arrival,
    replaying the pool of planted batches in turn.  Old slices keep their
    ids (the pool's old ids exist by the time a batch is replayed); new
    slices are renumbered to follow the stream's current slice count."""
    import numpy as np
    reqs = [Request(stream=s, arrival=0.0, kind="init", slice_ids=b0.slice_ids.numpy(),
                    row_ptr=b0.row_ptr.numpy(), X=b0.X, init_iters=init_iters, rows=b0.n_rows)]
    K = K0
    i = 0
    for (t_arr, s2, _) in load.arrivals:
        if s2 != s:
            continue
        b = pool[i % len(pool)]
        i += 1
        ids = b.slice_ids.numpy().copy()
        new = ids >= b.K_before
        ids[new] = K + (ids[new] - b.K_before)
        K += b.n_new
        reqs.append(Request(stream=s, arrival=t_arr, kind="update", slice_ids=ids,
                            row_ptr=b.row_ptr.numpy(), X=b.X, rows=b.n_rows))
    return reqs, K


def run_serving(a):
    """Serving loop (paper_2305_18376_gb300.serving) over the serving workload
    (synth.serving): independent planted streams, update batches arriving as
    one Poisson process.  Each stream's update batches come from a pool of
    three planted batches generated on the device and replayed in turn.
    Initial fits run first, untimed; the updates are then served in real
    time.  Reports the latency (arrival to completion) and rows/s of the
    updates, for the mixed and the FP64 paths."""
    import numpy as np
    import torch

    from paper_2305_18376_gb300.serving import Request, ServingLoop, latency_summary
    from synth.planted import PlantedStream, scaled
    from synth.serving import serving_load

    load = serving_load(n_streams=a.serve_streams, duration=a.serve_seconds, rate=a.serve_rate,
                        K0_range=(500, a.serve_k0_max))
    out = {"metric": "serving: update latency (arrival to completion) and rows/s",
           "streams": a.serve_streams, "arrivals": len(load.arrivals), "rate_per_s": a.serve_rate,
           "seconds": a.serve_seconds, "data": "synthetic",
           "config": {"workload": f"serving: {a.serve_streams} planted streams, J in (64, 128, 256), "
                                  f"R in (8, 16, 32), K0 in [500, {a.serve_k0_max}], Poisson arrivals "
                                  f"{a.serve_rate:g}/s for {a.serve_seconds:g} s, each batch touching a "
                                  "fraction U(0,1] of the slices with U{1..256} rows plus U{0..50} new "
                                  "slices; batches replayed from a pool of 3 per stream, device-resident"}}
    precs = [p for p in (("f16x3", torch.float32, "f32"), ("fp64", torch.float64, "f64"))
             if p[0] in a.serve_precisions.split(",")]
    for prec, tdt, idt in precs:
        specs, reqs_init, reqs_upd, V0 = {}, [], [], {}
        for s, w in enumerate(load.streams):
            ps = PlantedStream(scaled(w, steps=3), device="cuda", dtype=tdt)
            b0 = ps.batch(0)
            pool = [ps.batch(t) for t in range(1, 4)]
            reqs, K_end = _replay_requests(load, s, b0, pool, w.K0, tdt, Request, a.serve_init_iters)
            reqs_init.append(reqs[0])
            reqs_upd.extend(reqs[1:])
            specs[s] = dict(J=w.J, R=w.R, lam=w.lam, precision=prec, input_dtype=idt,
                            max_slices=K_end + 8,
                            max_rows=max([b0.n_rows] + [b.n_rows for b in pool]) + 16,
                            max_segments=max(b.slice_ids.numel() for b in [b0] + pool) + 8,
                            max_staged_rows=1)          # batches are device-resident: read in place
            V0[s] = np.random.default_rng(s).random((w.J, w.R))
        torch.cuda.synchronize()
        counters, profiles = {}, {}

        def prepare(s, m):
            m.set_factors(V0[s])
            if a.serve_profile:
                m.profile(True)

        def retire(s, m):
            V, W = m.factors()
            counters.setdefault(s, (m.counters(), m.K, float(np.abs(W).max()), float(np.abs(V).max())))
            if a.serve_profile:
                rep = m.profile_report()
                top = sorted(rep.items(), key=lambda kv: -kv[1][1])[:6]
                profiles[s] = {k: round(ms, 3) for k, (n, ms) in top}

        loop = ServingLoop(specs, int(a.serve_budget_gb * 1e9), max_inflight=max(2, a.serve_streams),
                           prepare=prepare, on_retire=retire)
        loop.run(reqs_init, realtime=False, final=False)   # fitted models stay for their updates
        torch.cuda.synchronize()
        loop.run(reqs_upd, realtime=True)
        summ = latency_summary(reqs_upd)
        summ["failed_requests"] = sum(1 for r in reqs_upd if r.failed)
        summ["failed_streams"] = sorted(loop.failed)
        summ["peak_resident_gb"] = loop.peak_resident / 1e9
        loop.close()
        # per stream: queueing (arrival to admission) against service (admission
        # to completion), and the numerical counters
        per = []
        for s, w in enumerate(load.streams):
            rs = [r for r in reqs_upd if r.stream == s and r.done is not None]
            if not rs:
                continue
            svc = np.array([r.done - r.admitted for r in rs]) * 1e3
            iss = np.array([r.issue_s for r in rs]) * 1e3
            lat = np.array([r.latency for r in rs]) * 1e3
            (timeouts, fallbacks), K_end, wmax, vmax = counters.get(s, ((None, None), None, None, None))
            per.append({"stream": s, "J": w.J, "R": w.R, "K0": w.K0, "K_end": K_end,
                        "updates": len(rs), "rows": int(sum(r.rows for r in rs)),
                        "service_ms_median": float(np.median(svc)), "service_ms_max": float(svc.max()),
                        "latency_ms_max": float(lat.max()), "issue_ms_median": float(np.median(iss)),
                        "issue_ms_max": float(iss.max()), "wait_timeouts": timeouts,
                        "fp64_fallback_solves": fallbacks, "max_abs_W": wmax, "max_abs_V": vmax,
                        "failed": loop.failed.get(s),
                        "profile_ms": profiles.get(s)})
        summ["per_stream"] = per
        out["mixed" if prec == "f16x3" else "fp64"] = summ
        del reqs_init, reqs_upd
        torch.cuda.empty_cache()
    print(json.dumps(out))


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.cycle_scan:
        run_cycle_scan(a)
    elif a.lambda_sweep:
        run_lambda_sweep(a)
    elif a.serving:
        # load every kernel at context creation, so that no request pays a
        # kernel's first-use load while others run
        os.environ.setdefault("CUDA_MODULE_LOADING", "EAGER")
        run_serving(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
