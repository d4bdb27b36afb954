"""Benchmark: forward+gradient spectra/s of the batched forward model and
log-likelihood on one GB300 (and N GPUs as independent shards, weak scaling).

A step is one es_forward_backward over the whole batch (every stage of the
path: setup, interpolation/extinction, chord optical depth / transit depth or
emission RT, binning, ln L, and the full adjoint). Inputs are resident in HBM
before the timed region; the per-step workspace (extinction, tau_bar,
alpha_bar: ~37 GB at the default workload) is far larger than L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   # the FP64 oracle on the host cores

Prints one JSON line (rank 0).
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

METRIC = "forward+gradient spectra/sec per GB300 (batched vs plain) at ≤1e-5 rel err vs FP64"
UNIT = "spectra/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="batched_trans")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain per-sample comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle cpu_baseline leg")
    ap.add_argument("--batch", type=int, default=None, help="override the workload's batch size")
    ap.add_argument("--no-tune", action="store_true", help="keep the built-in work-item sizes")
    ap.add_argument("--no-extra", action="store_true", help="skip the emission and high-resolution lines")
    ap.add_argument("--cpu-child", default=None, help=argparse.SUPPRESS)
    return ap.parse_args()


# --------------------------------------------------------------------------- CPU oracle timing
def oracle_sample_time(workload, n_sub, n_vec, seconds_cap=25.0):
    """Time the FP64 oracle (forward + complex-step gradient) on a bounded
    sample: the first `n_vec` valid parameter vectors of the workload on the
    first `n_sub` wavenumbers (same tables, layers, species). Returns seconds
    per full-resolution spectrum+gradient, scaled by N / n_sub."""
    from oracle import exoskry_oracle as O
    from paper_2602_19687_gb300 import synth
    w = synth.workload(workload, batch=max(8, n_vec * 4), n_nu=None)
    tabs = w.tables
    full_n = tabs.nu.size
    sub = synth.Tables(nu=tabs.nu[:n_sub], t_grid=tabs.t_grid, p_grid_bar=tabs.p_grid_bar,
                       log10_sigma=tabs.log10_sigma[..., :n_sub], cia_t_grid=tabs.cia_t_grid,
                       cia_h2h2=tabs.cia_h2h2[:, :n_sub], cia_h2he=tabs.cia_h2he[:, :n_sub])
    if w.table_dtype == "bf16":
        sub.log10_sigma = O.bf16_row_dequantized(sub.log10_sigma)
    lam_sub = 1e4 / sub.nu
    keep = (w.bin_hi_um <= lam_sub.max()) & (w.bin_lo_um >= lam_sub.min())
    lo, hi = w.bin_lo_um[keep], w.bin_hi_um[keep]
    mem = O.bin_members(sub.nu, lo, hi)
    m = w.model
    done, t0 = 0, time.perf_counter()
    for b in range(w.theta.shape[0]):
        kind = int(w.kind[b])
        th = m.full_theta(w.theta[b])[0]
        if not O.atmosphere(m, th)["valid"]:
            continue
        O.loglike_gradient(m, sub, th, kind, mem, w.y_obs[kind][keep], w.sigma[kind][keep],
                           list(m.free_idx))
        done += 1
        if done >= n_vec or time.perf_counter() - t0 > seconds_cap:
            break
    dt = time.perf_counter() - t0
    return dt / max(done, 1) * (full_n / n_sub), done, full_n


def cpu_baseline(workload, n_sub=1500, n_vec=2):
    """Run the oracle timing in a child process pinned to one thread."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-child", "%s:%d:%d" % (workload, n_sub, n_vec)]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=600)
    if r.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "error": r.stderr[-300:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": 1.0 / d["sec_per_spectrum"], "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d parameter vector(s) x first %d of %d wavenumbers, forward + complex-step gradient "
                      "(%s), scaled to a full spectrum; host cores available %d"
                      % (d["done"], n_sub, d["full_n"], workload, os.cpu_count() or 0)}


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r.split(",") for r in out.strip().splitlines() if r.strip()]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 4 + k and r[4 + k].strip().lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------- roofline
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def measure_nested(device, n_live=1000, batch=100, walk_steps=5, iterations=6, seed=3):
    """The batched nested sampler as the likelihood's consumer: a short run
    (fixed iteration count) on the batched transmission workload's model and
    tables with uniform priors, every call one es_set_batch + es_loglike on
    host vectors with the ln L read back. Parameter vectors per second over
    the whole run (sampler host work included) and the likelihood calls'
    share of it."""
    from paper_2602_19687_gb300 import binding, nested, synth
    w = synth.workload("batched_trans", batch=8)
    m = w.model
    ctx = binding.context_for(w, device=device)
    like = binding.LogLikeBatch(ctx, kind=0)
    ranges = synth.prior_ranges(m)
    lo = np.array([ranges[k][0] for k in m.free_idx])
    hi = np.array([ranges[k][1] for k in m.free_idx])
    rng = np.random.default_rng(seed)
    for b in (n_live, batch, batch, batch):   # warm-up: graph capture for both batch shapes
        like(lo + (hi - lo) * rng.random((b, lo.size)))
    spent = [0.0]

    def timed(theta):
        t = time.perf_counter()
        out = like(theta)
        spent[0] += time.perf_counter() - t
        return out

    t0 = time.perf_counter()
    res = nested.run(timed, lambda u: lo + (hi - lo) * u, lo.size, n_live=n_live, batch=batch,
                     walk_steps=walk_steps, max_iterations=iterations, seed=seed)
    dt = time.perf_counter() - t0
    ctx.es_destroy()
    return {"workload": "batched nested sampling on the batched_trans model (%d live points, %d replaced "
                        "per iteration, %d walk steps, %d iterations), ln L through host buffers"
                        % (n_live, batch, walk_steps, res.iterations),
            "value": res.evaluations / dt, "unit": "parameter vectors/s", "calls": res.calls,
            "evaluations": res.evaluations, "ms_per_call": 1e3 * spent[0] / res.calls,
            "likelihood_share": spent[0] / dt}


def kernel_work(name, w, n_valid):
    """Algorithmic work of one launch of each kernel at this workload:
    (amount, unit, bound), counted per kernel below."""
    from paper_2602_19687_gb300 import synth
    m = w.model
    B, L, S, N = n_valid, m.n_layers, m.n_species, w.tables.nu.size
    tri = L * (L + 1) // 2
    n_t = int(np.sum((w.kind == 0)[:B])) if B else 0
    n_e = B - n_t
    cloud = 1 if m.cloud_kind == synth.CLOUD_KH18 else 0
    if name in ("k_emis_fwd", "k_emis_bwd"):
        # per (emission vector, layer, wavenumber): the interpolation's S + 2
        # exponentials, one attenuation per Gauss-Legendre angle (4) and the
        # Planck function at the level (1); the adjoint recomputes all of them.
        # The non-grey cloud's second column adds 4 attenuations.
        return n_e * L * (S + 7 + 4 * cloud) * N, "ex2", "alu"
    if name == "k_trans_fwd":
        # one ex2 per (vector, layer, species or CIA pair, wavenumber) of the
        # interpolation, plus exp(-tau_i) per (vector, impact parameter,
        # wavenumber), twice with the non-grey cloud (clear and cloudy chords)
        return n_t * L * (S + 3 + cloud) * N, "ex2", "alu"
    if name == "k_trans_bwd":
        # the adjoint recomputes the interpolation's exponentials (and the
        # cloudy chord's transmission)
        return n_t * L * (S + 2 + cloud) * N, "ex2", "alu"
    return None


def measured_traffic(name, n_vectors):
    """DRAM bytes per launch of `name` from the committed ncu capture, scaled
    from its batch to n_vectors transmission vectors; None when the kernel
    sources changed since the capture."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic_k_trans_b128.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    for rel, digest in d["sources_sha256"].items():
        with open(os.path.join(ROOT, rel), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != digest:
                return None
    b = d["dram_bytes_per_launch"].get(name)
    return None if b is None else b * n_vectors / d["capture_vectors"]


def alu_peak(kind, sm_mhz):
    """Peaks from unit counts x clock (152 SMs): MUFU ex2 32/clk/SM on
    GB300; FP32 FMA 128 lanes x 2 flop/clk/SM."""
    clk = sm_mhz * 1e6
    if kind == "ex2":
        return 152 * 32 * clk
    if kind == "flop":
        return 152 * 128 * 2 * clk
    return None


# --------------------------------------------------------------------------- main arms
# --------------------------------------------------------------------------- other workloads
def measure_workload(name, device, steps=5, warmup=3):
    """Forward+gradient throughput of another synthetic workload (graph
    replay, device-resident inputs, CUDA events): spectra/s and ms/step."""
    import torch
    from paper_2602_19687_gb300 import binding, synth
    w = synth.workload(name)
    ctx = binding.context_for(w, device=device)
    dev = torch.device("cuda", device)
    B = w.theta.shape[0]
    th = torch.tensor(w.theta, dtype=torch.float64, device=dev)
    ctx.es_set_batch(th, torch.tensor(w.kind, dtype=torch.int32, device=dev))
    lnl = torch.empty(B, dtype=torch.float64, device=dev)
    grad = torch.empty_like(th)
    ctx.es_autotune()
    for _ in range(warmup):
        ctx.es_forward_backward(lnl, grad)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream(dev)
    e0.record(stream)
    for _ in range(steps):
        ctx.es_forward_backward(lnl, grad)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    n_em = int(np.sum(w.kind == 1))
    ctx.es_destroy()
    return {"workload": name + ": " + w.description, "vectors": B, "emission_vectors": n_em,
            "value": B / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps, "warmup": warmup}


# --------------------------------------------------------------------------- sharding
def shard_seed(rank):
    """Each rank evaluates its own batch of parameter vectors (weak scaling:
    independent shards, no data-path collective)."""
    return 42 + rank


def max_over_ranks(x, world, device):
    """The slowest rank's time: all-reduce MAX (identity at world == 1)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(batch_per_rank, world, ms_max):
    """Whole-job spectra/s: the units all ranks processed over the slowest rank's time."""
    return batch_per_rank * world / (ms_max / 1e3)


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2602_19687_gb300 import binding, synth
    import __graft_entry__

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
        __graft_entry__.build()

    def barrier():
        if world > 1:
            dist.barrier()

    w = synth.workload(args.workload, batch=args.batch, seed=shard_seed(rank))   # each rank: its own shard
    ctx = binding.context_for(w, device=local)
    B = w.theta.shape[0]
    nfree = w.theta.shape[1]
    theta = torch.tensor(w.theta, dtype=torch.float64, device=dev)
    kind = torch.tensor(w.kind, dtype=torch.int32, device=dev)
    ctx.es_set_batch(theta, kind)
    lnl = torch.empty(B, dtype=torch.float64, device=dev)
    grad = torch.empty((B, nfree), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    tuned = ctx.es_autotune() if not args.no_tune else (0, 0)   # work-item sizes, outside the timed region
    for _ in range(args.warmup):
        ctx.es_forward_backward(lnl, grad)
    torch.cuda.synchronize(dev)
    flags = torch.empty(B, dtype=torch.int32, device=dev)
    ctx.es_get_flags(flags)
    n_valid = int((flags == 0).sum().item())

    # ---- timed region (device-resident inputs; the step replays its CUDA graph)
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    launches = 0
    for _ in range(args.steps):
        ctx.es_forward_backward(lnl, grad)
        launches += ctx.es_query(7)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()

    # ---- the same steps launched directly with per-kernel CUDA events (for
    # the roofline and the kernel shares; profiling turns graph replay off)
    ctx.es_set_profiling(True)
    torch.cuda.synchronize(dev)
    ep0, ep1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ep0.record(stream)
    for _ in range(args.steps):
        ctx.es_forward_backward(lnl, grad)
    ep1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    ms_profiled = ep0.elapsed_time(ep1) / args.steps
    prof = ctx.es_get_profile()
    ctx.es_set_profiling(False)
    ms_max = max_over_ranks(ms, world, dev)
    value = job_throughput(B, world, ms_max)

    # ---- end to end through the C ABI with host buffers (pinned)
    th_host = torch.tensor(w.theta, dtype=torch.float64).pin_memory().numpy()
    kd_host = np.ascontiguousarray(w.kind, np.int32)
    lnl_h = torch.empty(B, dtype=torch.float64).pin_memory().numpy()
    grad_h = torch.empty((B, nfree), dtype=torch.float64).pin_memory().numpy()
    ctx.es_set_batch(th_host, kd_host)
    ctx.es_forward_backward(lnl_h, grad_h)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.es_set_batch(th_host, kd_host)
        ctx.es_forward_backward(lnl_h, grad_h)
    t1 = time.perf_counter()
    barrier()
    e2e_ms = (t1 - t0) * 1e3 / args.steps
    e2e_value = job_throughput(B, world, max_over_ranks(e2e_ms, world, dev))

    # ---- roofline of the dominant kernel (live CUDA-event times)
    peaks, peak_src = measured_peaks()
    ex2_rate, ffma2_rate = binding.probe_rates(local)
    sm_mhz = (clk or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    per_kernel = {}
    total_prof = sum(p[1] for p in prof) or 1.0
    for name, tot, n in prof:
        per_kernel[name] = {"ms_per_launch": tot / max(n, 1), "launches": n, "share": tot / total_prof}
    top = max(prof, key=lambda p: p[1])[0] if prof else None
    roof = None
    if top is not None:
        wk = kernel_work(top, w, n_valid)
        ms_launch = per_kernel[top]["ms_per_launch"]
        if wk is not None:
            amount, unit_kind, bound = wk
            achieved = amount / (ms_launch / 1e3)
            peak = ex2_rate if unit_kind == "ex2" else alu_peak(unit_kind, sm_mhz)
            scale = 1e12
            roof = {"kernel": top, "bound": bound, "achieved": achieved / scale,
                    "peak": peak / scale if peak else None,
                    "unit": "T%s/s" % unit_kind, "frac": (achieved / peak) if peak else None,
                    "traffic": measured_traffic(top, int(np.sum(w.kind[:n_valid] == 0))),
                    "traffic_unit": "bytes per launch (ncu capture at B=128, scaled by vectors)",
                    "ms_per_launch": ms_launch,
                    "peak_source": ("measured: es_probe_rates MUFU ex2 throughput on this GPU"
                                    if unit_kind == "ex2" else
                                    "derived from unit counts x median SM clock %.0f MHz" % sm_mhz),
                    "nominal_peak": alu_peak(unit_kind, sm_mhz) / scale if alu_peak(unit_kind, sm_mhz) else None}

    # ---- plain per-sample path (batched vs plain): the plain JWST-shaped
    # workload, and the batched workload itself one vector per call
    def plain_ms(wp, theta_row, kind_row):
        cp = binding.context_for(wp, device=local)
        thp = torch.tensor(theta_row, dtype=torch.float64, device=dev)
        cp.es_set_batch(thp, torch.tensor(kind_row, dtype=torch.int32, device=dev))
        lp = torch.empty(1, dtype=torch.float64, device=dev)
        gp = torch.empty_like(thp)
        for _ in range(3):
            cp.es_forward_backward(lp, gp)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 20
        e0.record(stream)
        for _ in range(reps):
            cp.es_forward_backward(lp, gp)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        cp.es_destroy()
        return e0.elapsed_time(e1) / reps

    plain = plain_same = None
    if not args.no_plain and rank == 0:
        wp = synth.workload("jwst_plain")
        pms = plain_ms(wp, wp.theta, wp.kind)
        plain = {"value": 1e3 / pms, "unit": UNIT, "ms_per_spectrum": pms,
                 "workload": "jwst_plain: " + wp.description + " (one vector per call, forward+gradient)"}
        pms = plain_ms(w, w.theta[:1], w.kind[:1])
        plain_same = {"value": 1e3 / pms, "unit": UNIT, "ms_per_spectrum": pms,
                      "workload": args.workload + ": " + w.description +
                      " (one vector per call, forward+gradient)"}

    extra = None
    if rank == 0 and not args.no_extra:
        extra = [measure_workload(n, local) for n in ("batched_emis", "highres", "browndwarf", "cloudy_trans", "cloudy_emis")]
        extra.append(measure_nested(local))
    cpu = cpu_baseline(args.workload) if (rank == 0 and not args.no_cpu) else None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded tables, data and parameter batches)",
            "config": {"workload": args.workload + ": " + w.description, "batch_per_gpu": B,
                       "valid_vectors": n_valid, "n_nu": int(w.tables.nu.size), "layers": w.model.n_layers,
                       "species": w.model.n_species, "free_params": nfree, "tables": w.table_dtype,
                       "l2": "inputs larger than L2 (per-step workspace ~%.0f GB)" % (ctx.es_query(6) / 1e9),
                       "parallelism": "independent shards, one process per GPU"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(B * nfree * 8 + B * 4),
                    "d2h_bytes_per_step": int(B * 8 + B * nfree * 8)},
            "gpu_launches": int(launches),
            "graph_replay": bool(ctx.es_query(10)),
            "work_item_tiles": {"k_trans_fwd": tuned[0], "k_trans_bwd": tuned[1]},
            "ms_per_step_direct_launches": ms_profiled,
            "roofline": roof,
            "kernels": per_kernel,
            "plain": plain,
            "batched_over_plain": (value / world / plain["value"]) if plain else None,
            "plain_same_workload": plain_same,
            "batched_over_plain_same_workload": (value / world / plain_same["value"]) if plain_same else None,
            "cpu_baseline": cpu,
            "other_workloads": extra,
            "clocks": clk,
            "peaks_source": peak_src,
            "probe": {"ex2_per_s": ex2_rate, "ffma2_per_s": ffma2_rate},
        }
        print(json.dumps(line))
    ctx.es_destroy()
    if world > 1:
        dist.destroy_process_group()


def run_reference(args):
    """The FP64 oracle as it stands, timed on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    per = []
    for _ in range(args.warmup + args.steps):
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1")
        cmd = [sys.executable, os.path.abspath(__file__), "--cpu-child", "%s:%d:%d" % (args.workload, 600, 1)]
        r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=600)
        if r.returncode != 0:
            raise RuntimeError("oracle timing child failed: " + r.stderr[-500:])
        d = json.loads(r.stdout.strip().splitlines()[-1])
        per.append(d["sec_per_spectrum"])
    timed = per[args.warmup:]
    sps = 1.0 / float(np.mean(timed))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": sps, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(timed)) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": args.workload},
        "cpu_baseline": {"value": sps, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "per step: 1 parameter vector x first 600 wavenumbers, forward + "
                                   "complex-step gradient, scaled to a full spectrum"},
        "e2e": {"value": sps, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def main():
    args = parse()
    if args.cpu_child:
        name, n_sub, n_vec = args.cpu_child.split(":")
        sec, done, full_n = oracle_sample_time(name, int(n_sub), int(n_vec))
        print(json.dumps({"sec_per_spectrum": sec, "done": done, "full_n": full_n}))
        return
    if args.impl == "reference":
        run_reference(args)
        return
    run_gpu(args)


if __name__ == "__main__":
    main()
