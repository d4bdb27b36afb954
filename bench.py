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
    ap.add_argument("--oracle-vectors", type=int, default=None,
                    help="parameter vectors the cpu_baseline leg runs through the oracle (default: host cores)")
    return ap.parse_args()


# --------------------------------------------------------------------------- the oracle on the host cores
# The FP64 oracle runs in a process pool (spawn) over all host cores, on whole
# spectra: one task is the forward model of one parameter vector, or the
# complex-step derivative of its ln L with respect to one free parameter, so
# the n_free + 1 tasks of a vector's forward + gradient run in parallel. It is
# used by the cpu_baseline leg and by the reference arm only. Its FP64-table
# outputs are also what the BF16-table GPU path's error is measured against.
_ORACLE_CACHE = {}


def _oracle_setup(key, tables):
    from oracle import exoskry_oracle as O
    from paper_2602_19687_gb300 import synth
    if key not in _ORACLE_CACHE:
        name, batch, seed = key[:3]
        w = synth.workload(name, batch=batch, seed=seed, n_nu=key[3] if len(key) > 3 else None)
        _ORACLE_CACHE[key] = {"w": w, "mem": O.bin_members(w.tables.nu, w.bin_lo_um, w.bin_hi_um)}
    ent = _ORACLE_CACHE[key]
    if tables == "bf16" and "bf16" not in ent:
        w = ent["w"]
        t = synth.Tables(**{f: getattr(w.tables, f) for f in ("nu", "t_grid", "p_grid_bar", "log10_sigma",
                                                             "cia_t_grid", "cia_h2h2", "cia_h2he")})
        t.log10_sigma = O.bf16_row_dequantized(w.tables.log10_sigma)
        ent["bf16"] = t
    return ent["w"], ent["mem"], (ent["bf16"] if tables == "bf16" else ent["w"].tables)


def oracle_task(task):
    """task = (workload key (name, batch, seed[, n_nu]), vector index, tables, slot):
    slot None is the forward model (native spectrum, binned model, ln L);
    slot k the complex-step derivative of ln L with respect to free parameter
    k. tables "fp64": the synthetic tables as generated; "bf16": the values
    the BF16 storage holds (row offset + rounded residual)."""
    from oracle import exoskry_oracle as O
    key, b, tables, slot = task
    w, mem, tabs = _oracle_setup(key, tables)
    m = w.model
    th = m.full_theta(w.theta[b])[0]
    kind = int(w.kind[b])
    y, sig = w.y_obs[kind], w.sigma[kind]
    t0 = time.perf_counter()
    if slot is None:
        out = O.forward(m, tabs, th, kind, mem)
        if out is None:
            res = {"valid": False, "lnl": O.INVALID_LNL}
        else:
            res = {"valid": True, "spec": out[0], "binned": out[1],
                   "lnl": O.log_likelihood(out[1], y, sig, th[m.n_species + O.P_C_INFL])}
    else:
        res = {"grad": float(O.loglike_gradient(m, tabs, th, kind, mem, y, sig, [m.free_idx[slot]])[0])}
    res.update(key=key, b=b, tables=tables, slot=slot, seconds=time.perf_counter() - t0)
    return res


REF_VECTORS = 4   # parameter vectors per step of the reference arm


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_pool(n=None):
    import multiprocessing as mp
    n = n or host_cores()
    env = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1"}
    os.environ.update(env)   # one thread per worker: the pool supplies the parallelism
    return mp.get_context("spawn").Pool(n), n


def valid_vectors(w, count):
    """The first `count` parameter vectors the oracle's own profile,
    chemistry and hydrostatics accept."""
    from oracle import exoskry_oracle as O
    out = []
    for b in range(w.theta.shape[0]):
        if O.atmosphere(w.model, w.model.full_theta(w.theta[b])[0])["valid"]:
            out.append(b)
            if len(out) == count:
                break
    return out


def oracle_gradients(pool, key, vectors, nfree, tables="fp64"):
    """Forward + gradient of each vector on whole spectra over the pool:
    (per-vector results, wall seconds)."""
    tasks = [(key, b, tables, None) for b in vectors] + [(key, b, tables, k) for b in vectors for k in range(nfree)]
    t0 = time.perf_counter()
    res = pool.map(oracle_task, tasks, chunksize=1)
    wall = time.perf_counter() - t0
    out = {b: {"grad": np.zeros(nfree)} for b in vectors}
    for r in res:
        if r["slot"] is None:
            out[r["b"]].update({k: v for k, v in r.items() if k in ("valid", "spec", "binned", "lnl")})
        else:
            out[r["b"]]["grad"][r["slot"]] = r["grad"]
    return out, wall


def oracle_forwards(pool, key, vectors, tables):
    res = pool.map(oracle_task, [(key, b, tables, None) for b in vectors], chunksize=1)
    return {r["b"]: r for r in res}


def cpu_baseline(pool, cores, key, vectors, nfree):
    """The oracle as it stands, timed on the host cores: forward + complex-step
    gradient of whole spectra for `vectors` (one pool task per vector and per
    gradient slot). Returns (cpu_baseline record, oracle outputs)."""
    out, wall = oracle_gradients(pool, key, vectors, nfree)
    rec = {"value": len(vectors) / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
           "seconds": wall,
           "sample": "%d parameter vectors of %s (seed %d), whole spectra (all wavenumbers), forward + "
                     "complex-step gradient of ln L in %d free parameters, FP64 on the unquantized tables; "
                     "one task per vector and gradient slot over a %d-process pool"
                     % (len(vectors), key[0], key[2], nfree, cores)}
    return rec, out


def _rel(a, b, floor=0.0):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), floor)


def _stats(x):
    x = np.asarray(x, np.float64).ravel()
    return {"max": float(np.max(x)), "median": float(np.median(x))} if x.size else None


def bf16_error(gpu, ref, ref_bf16=None):
    """Error of the GPU path (BF16 tables, FP32 arithmetic) against the FP64
    oracle on the unquantized tables, over the sampled vectors: native
    spectrum and binned model (relative), ln L (absolute and relative), and
    the gradient per component (relative, components smaller than 1e-3 of the
    vector's largest measured against that floor; and in units of the
    gradient parity tolerance 1e-3 |ref| + 1e-4 max |ref|). With ref_bf16 (the oracle
    on the BF16-stored table values) also the GPU arithmetic's own error."""
    vecs = [b for b in ref if ref[b].get("valid")]
    out = {"vectors": len(vecs)}
    if not vecs:
        return out
    out["native"] = _stats(np.concatenate([_rel(gpu["spec"][b], ref[b]["spec"]) for b in vecs]))
    out["binned"] = _stats(np.concatenate([_rel(gpu["binned"][b], ref[b]["binned"]) for b in vecs]))
    dl = np.array([gpu["lnl"][b] - ref[b]["lnl"] for b in vecs])
    out["lnl_abs"] = _stats(np.abs(dl))
    out["lnl_rel"] = _stats(np.abs(dl) / np.abs([ref[b]["lnl"] for b in vecs]))
    gv = [b for b in vecs if b in gpu.get("grad", {}) and "grad" in ref[b]]
    if gv:
        g = [_rel(gpu["grad"][b], ref[b]["grad"], 1e-3 * np.max(np.abs(ref[b]["grad"]))) for b in gv]
        out["grad"] = _stats(np.concatenate(g))
        # in units of the gradient parity tolerance, 1e-3 |ref| + 1e-4 max |ref| (1 = at the tolerance)
        t = [np.abs(gpu["grad"][b] - ref[b]["grad"]) /
             (1e-3 * np.abs(ref[b]["grad"]) + 1e-4 * np.max(np.abs(ref[b]["grad"]))) for b in gv]
        out["grad_over_tolerance"] = _stats(np.concatenate(t))
        out["grad_vectors"] = len(gv)
    if ref_bf16:
        v2 = [b for b in ref_bf16 if ref_bf16[b].get("valid")]
        if v2:
            out["gpu_arithmetic_only"] = {
                "native": _stats(np.concatenate([_rel(gpu["spec"][b], ref_bf16[b]["spec"]) for b in v2])),
                "lnl_abs": _stats(np.abs([gpu["lnl"][b] - ref_bf16[b]["lnl"] for b in v2]))}
    return out


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
    if name in ("k_eaa_ext", "k_eaa_abar"):
        # delta-EAA: the interpolation's S + 2 exponentials per (emission
        # vector, layer, wavenumber), stored (ext) or recomputed (abar)
        return n_e * L * (S + 2) * N, "ex2", "alu"
    if name == "k_eaa_rt":
        # delta-EAA RT per column (clear, and cloudy with the non-grey cloud)
        # and layer: going up, 4 zeroth-order attenuations and the Planck
        # value; going down, 4 zeroth-order and 4 first-order attenuations
        return n_e * L * 13 * (1 + cloud) * N, "ex2", "alu"
    if name == "k_eaa_rt_bwd":
        # its adjoint: the forward's 13 and, in the third pass, 4 zeroth-order
        # attenuations and dB/dT at the level
        return n_e * L * 18 * (1 + cloud) * N, "ex2", "alu"
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


def emission_fp32_ops(name, w, n_valid):
    """Algorithmic FP32 operations (an FMA counts as one) of one launch of an
    emission kernel, per (emission vector, layer, wavenumber): 4 per species
    (the bilinear exponent in coefficient form, 3, and its sum), 6 for the
    two CIA pairs, the number density and Rayleigh, 1 for dtau = alpha dr, 3
    for the Planck function at the level and 7 per flux angle for the
    linear-in-tau step (x = dtau/mu, 1 - E, the linear-source factor and the
    intensity update): 4 S + 10 + 7 n_mu. The adjoint counts three times the
    forward's (the recompute plus two operations per forward operation for
    the reverse sweep). The non-grey cloud's second column adds 7 n_mu + 1."""
    from paper_2602_19687_gb300 import synth
    m = w.model
    n_e = int(np.sum((w.kind == 1)[:n_valid]))
    cloud = 1 if m.cloud_kind == synth.CLOUD_KH18 else 0
    per = 4 * m.n_species + 10 + 7 * 4 + cloud * (7 * 4 + 1)
    ops = n_e * m.n_layers * w.tables.nu.size * per
    return ops * (3 if name == "k_emis_bwd" else 1)


def trans_fp32_ops(name, w, n_valid):
    """Algorithmic FP32 operations (an FMA counts as one) of one launch of a
    transmission kernel, per (transmission vector, layer, wavenumber).
    Forward: 4 per species (the bilinear exponent in coefficient form, 3, and
    its sum), 4 for the two CIA pairs, 3 to assemble alpha (number density,
    Rayleigh, the lane pair's sum), 1 for the BF16 residual of the split
    operand, and 3 per impact parameter in the epilogue (exponent argument,
    1 - exp(-tau), area weight): 4 S + 11. Adjoint: the forward's 4 S + 4
    recompute, 2 per species for the per-species and temperature-slope sums,
    9 for the per-layer reduction inputs (alpha_bar n, the CIA products and
    the four values), 3 to assemble alpha and 4 per impact parameter in the
    tau_bar phase (dbar A exp(-tau) and the area sum): 6 S + 20. The chord
    products run on the tensor cores and are not counted here."""
    m = w.model
    n_t = int(np.sum((w.kind == 0)[:n_valid]))
    S = m.n_species
    per = 4 * S + 11 if name == "k_trans_fwd" else 6 * S + 20
    return n_t * m.n_layers * w.tables.nu.size * per


def measured_traffic(name, n_vectors):
    """DRAM bytes per launch of `name` from the committed ncu captures
    (profiles/traffic_k_trans.json: one capture per batch size), scaled from
    the capture with the batch nearest to n_vectors transmission vectors;
    None when the kernel sources changed since the captures."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic_k_trans.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    for rel, digest in d["sources_sha256"].items():
        with open(os.path.join(ROOT, rel), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != digest:
                return None
    caps = [c for c in d["captures"] if name in c["dram_bytes_per_launch"]]
    if not caps:
        return None
    c = min(caps, key=lambda c: abs(c["vectors"] - n_vectors))
    return c["dram_bytes_per_launch"][name] * n_vectors / c["vectors"]


def measured_alpha_traffic(workload):
    """DRAM bytes per launch of the one-vector opacity stage on `workload`
    from the committed ncu capture (profiles/traffic_k_trans_alpha.json);
    None for another workload or when the kernel sources changed since."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic_k_trans_alpha.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("workload") != workload:
        return None
    for rel, digest in d["sources_sha256"].items():
        with open(os.path.join(ROOT, rel), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != digest:
                return None
    return d["dram_bytes_per_launch"]


def measured_instructions(name, n_vectors, n_layers, n_nu, record="instructions_k_trans.json"):
    """Warp instructions per launch of `name` from a committed ncu capture
    (profiles/instructions_k_trans.json for the transmission kernels,
    profiles/instructions_k_eaa.json for the delta-EAA kernels: per (vector,
    layer, 32 wavenumbers)), scaled to n_vectors x n_layers x n_nu; None when
    the kernel sources changed since the capture."""
    import hashlib
    p = os.path.join(ROOT, "profiles", record)
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    for rel, digest in d["sources_sha256"].items():
        with open(os.path.join(ROOT, rel), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != digest:
                return None
    if name not in d["per_unit"]:
        return None
    return d["per_unit"][name] * n_vectors * n_layers * n_nu / 32.0


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
def measure_workload(name, device, steps=5, warmup=3, out_vectors=None, probe=None, sm_mhz=2070.0):
    """Forward+gradient and forward-only throughput of another synthetic
    workload (graph replay, device-resident inputs, CUDA events): spectra/s
    and ms/step; per-kernel times of two directly launched steps (with the
    emission kernels' roofline when they run); and, for `out_vectors`, the
    GPU's native spectrum, binned model, ln L and gradient (for the error
    against the FP64 oracle)."""
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
    stream = torch.cuda.current_stream(dev)

    def timed(call):
        for _ in range(warmup):
            call()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            call()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / steps

    ms = timed(lambda: ctx.es_forward_backward(lnl, grad))
    ms_fwd = timed(lambda: ctx.es_loglike(lnl))
    ctx.es_set_profiling(True)
    for _ in range(2):
        ctx.es_forward_backward(lnl, grad)
    torch.cuda.synchronize(dev)
    prof = ctx.es_get_profile()
    ctx.es_set_profiling(False)
    flags = torch.empty(B, dtype=torch.int32, device=dev)
    ctx.es_forward_backward(lnl, grad)
    ctx.es_get_flags(flags)
    n_valid = int((flags == 0).sum().item())
    kernels = {k: {"ms_per_launch": t / max(n, 1), "launches": n} for k, t, n in prof}
    roof = {}
    for k in ("k_emis_fwd", "k_emis_bwd"):
        if k in kernels and probe:
            sec = kernels[k]["ms_per_launch"] / 1e3
            ex2 = kernel_work(k, w, B)[0] / sec
            fp32 = emission_fp32_ops(k, w, B) / sec
            roof[k] = {"bound": "alu", "ms_per_launch": kernels[k]["ms_per_launch"],
                       "ex2": {"achieved": ex2 / 1e12, "peak": probe[0] / 1e12, "unit": "Tex2/s",
                               "frac": ex2 / probe[0]},
                       "fp32": {"achieved": fp32 / 1e12, "peak": 2 * probe[1] / 1e12, "unit": "Top/s",
                                "frac": fp32 / (2 * probe[1]),
                                "peak_source": "measured: es_probe_rates packed FFMA2 rate x 2 lanes"}}
    for k in ("k_eaa_ext", "k_eaa_rt", "k_eaa_rt_bwd", "k_eaa_abar"):
        if k in kernels and probe:
            sec = kernels[k]["ms_per_launch"] / 1e3
            # the forward kernels run every emission vector, the adjoint ones the valid vectors
            nvec = B if k in ("k_eaa_ext", "k_eaa_rt") else n_valid
            ex2 = kernel_work(k, w, nvec)[0] / sec
            roof[k] = {"bound": "alu", "ms_per_launch": kernels[k]["ms_per_launch"],
                       "ex2": {"achieved": ex2 / 1e12, "peak": probe[0] / 1e12, "unit": "Tex2/s",
                               "frac": ex2 / probe[0]}}
            inst = measured_instructions(k, nvec, w.model.n_layers, w.tables.nu.size, "instructions_k_eaa.json")
            if inst is not None and name == "scattering_emis":
                # warp instructions against one per clock per SM sub-partition at the median SM clock
                ipeak = 152 * 4 * sm_mhz * 1e6
                roof[k]["issue"] = {"achieved": inst / sec / 1e12, "peak": ipeak / 1e12,
                                    "unit": "T warp-instructions/s", "frac": inst / sec / ipeak,
                                    "instructions_per_launch": inst,
                                    "count_source": "profiles/instructions_k_eaa.json (ncu, same sources)"}
    gpu_out = None
    if out_vectors:
        N, nb = w.tables.nu.size, w.bin_lo_um.size
        spec = torch.empty((B, N), dtype=torch.float32, device=dev)
        binned = torch.empty((B, nb), dtype=torch.float64, device=dev)
        lnl_f = torch.empty(B, dtype=torch.float64, device=dev)
        ctx.es_forward(spectrum=spec, binned=binned, lnl=lnl_f)
        torch.cuda.synchronize(dev)
        idx = list(out_vectors)
        gpu_out = {"spec": dict(zip(idx, spec[idx].cpu().numpy().astype(np.float64))),
                   "binned": dict(zip(idx, binned[idx].cpu().numpy())),
                   "lnl": dict(zip(idx, lnl_f[idx].cpu().numpy())),
                   "grad": dict(zip(idx, grad[idx].cpu().numpy()))}
    n_em = int(np.sum(w.kind == 1))
    ctx.es_destroy()
    rec = {"workload": name + ": " + w.description, "vectors": B, "emission_vectors": n_em,
           "valid_vectors": n_valid, "value": B / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
           "forward_only": {"value": B / (ms_fwd / 1e3), "unit": "spectra/s (ln L only)", "ms_per_step": ms_fwd},
           "kernels": kernels, "steps": steps, "warmup": warmup}
    if roof:
        rec["roofline"] = roof
    return rec, w, gpu_out


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
    tuned = ctx.es_autotune() if not args.no_tune else ctx.launch_shapes()   # outside the timed region
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

    # ---- forward only (ln L, the sampler's call): graph replay, device buffers
    ctx.es_set_batch(theta, kind)
    for _ in range(args.warmup):
        ctx.es_loglike(lnl)
    torch.cuda.synchronize(dev)
    barrier()
    ef0, ef1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ef0.record(stream)
    for _ in range(args.steps):
        ctx.es_loglike(lnl)
    ef1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    fwd_ms = max_over_ranks(ef0.elapsed_time(ef1) / args.steps, world, dev)
    forward_only = {"value": job_throughput(B, world, fwd_ms), "unit": "spectra/s (ln L only, es_loglike)",
                    "ms_per_step": fwd_ms}

    # ---- the GPU's outputs for the vectors the oracle legs sample (BF16-table error)
    gpu_head = None
    if rank == 0 and not args.no_cpu:
        sample = valid_vectors(w, args.oracle_vectors)
        spec_d = torch.empty((B, w.tables.nu.size), dtype=torch.float32, device=dev)
        bin_d = torch.empty((B, w.bin_lo_um.size), dtype=torch.float64, device=dev)
        lnl_d = torch.empty(B, dtype=torch.float64, device=dev)
        ctx.es_forward(spectrum=spec_d, binned=bin_d, lnl=lnl_d)
        ctx.es_forward_backward(lnl, grad)
        torch.cuda.synchronize(dev)
        gpu_head = {"spec": {b: spec_d[b].cpu().numpy().astype(np.float64) for b in sample},
                    "binned": {b: bin_d[b].cpu().numpy() for b in sample},
                    "lnl": {b: float(lnl_d[b]) for b in sample},
                    "grad": {b: grad[b].cpu().numpy() for b in sample}}
        del spec_d, bin_d

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
                    "traffic_unit": "bytes per launch (ncu capture at the nearest batch size, scaled by vectors)",
                    "ms_per_launch": ms_launch,
                    "peak_source": ("measured: es_probe_rates MUFU ex2 throughput on this GPU"
                                    if unit_kind == "ex2" else
                                    "derived from unit counts x median SM clock %.0f MHz" % sm_mhz),
                    "nominal_peak": alu_peak(unit_kind, sm_mhz) / scale if alu_peak(unit_kind, sm_mhz) else None}
            if top in ("k_trans_fwd", "k_trans_bwd"):
                # the launch's instruction issue: its warp instructions (committed ncu
                # count, scaled) against one warp instruction per clock per SM
                # sub-partition (4 per SM) at the median SM clock of the timed region
                n_t = int(np.sum(w.kind[:n_valid] == 0))
                inst = measured_instructions(top, n_t, w.model.n_layers, w.tables.nu.size)
                if inst is not None:
                    ipeak = 152 * 4 * sm_mhz * 1e6
                    ach = inst / (ms_launch / 1e3)
                    roof["issue"] = {"achieved": ach / 1e12, "peak": ipeak / 1e12, "unit": "T warp-instructions/s",
                                     "frac": ach / ipeak, "instructions_per_launch": inst,
                                     "peak_source": "152 SMs x 4 issue slots per clock x median SM clock %.0f MHz"
                                                    % sm_mhz,
                                     "count_source": "profiles/instructions_k_trans.json (ncu, same sources)"}
                # the same launch as FP32 operations against the probed packed-FMA rate
                ops = trans_fp32_ops(top, w, n_valid) / (ms_launch / 1e3)
                roof["fp32"] = {"achieved": ops / 1e12, "peak": 2 * ffma2_rate / 1e12, "unit": "Top/s",
                                "frac": ops / (2 * ffma2_rate),
                                "peak_source": "measured: es_probe_rates packed FFMA2 rate x 2 lanes"}

    # ---- plain per-sample path (batched vs plain): the plain JWST-shaped
    # workload, and the batched workload itself one vector per call
    def plain_ms(wp, theta_row, kind_row, roof=False):
        """ms per spectrum of the one-vector path: each step timed alone with
        CUDA events after an L2 flush (a step's working set fits in L2); with
        roof, the opacity stage's roofline: its algorithmic bytes (the raw
        table and CIA rows bracketing the vector's layers, es_query 17) over
        its per-launch duration in profiled steps, each after an L2 flush."""
        cp = binding.context_for(wp, device=local)
        thp = torch.tensor(theta_row, dtype=torch.float64, device=dev)
        cp.es_set_batch(thp, torch.tensor(kind_row, dtype=torch.int32, device=dev))
        lp = torch.empty(1, dtype=torch.float64, device=dev)
        gp = torch.empty_like(thp)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        for _ in range(3):
            cp.es_forward_backward(lp, gp)
        reps, tot = 20, 0.0
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            cp.es_forward_backward(lp, gp)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            tot += e0.elapsed_time(e1)
        rl = None
        if roof:
            cp.es_set_profiling(True)
            for _ in range(10):
                flush.zero_()
                cp.es_forward_backward(lp, gp)
            torch.cuda.synchronize(dev)
            prof = {k: t / max(n, 1) for k, t, n in cp.es_get_profile()}
            cp.es_set_profiling(False)
            cp.es_loglike(lp)
            nbytes = cp.es_query(17)
            ms_a = prof.get("k_trans_alpha")
            if ms_a and nbytes > 0:
                gbs = nbytes / (ms_a / 1e3) / 1e9
                hbm_peak = float(peaks["hbm_gbs"])
                rl = {"kernel": "k_trans_alpha", "bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                      "frac": gbs / hbm_peak, "algorithmic_bytes": nbytes, "ms_per_launch": ms_a,
                      "traffic": measured_alpha_traffic(wp.name),
                      "traffic_unit": "DRAM bytes per launch (ncu capture, same sources)",
                      "bytes_source": "raw table and CIA rows bracketing the vector's layers (es_query 17), "
                                      "each read once",
                      "timing": "CUDA events around the launch in profiled steps, L2 flushed before each step",
                      "peak_source": peak_src + " hbm_gbs (copy bandwidth)"}
        cp.es_destroy()
        return tot / reps, rl

    plain = plain_same = None
    if not args.no_plain and rank == 0:
        wp = synth.workload("jwst_plain")
        pms, rl = plain_ms(wp, wp.theta, wp.kind, roof=True)
        plain = {"value": 1e3 / pms, "unit": UNIT, "ms_per_spectrum": pms,
                 "workload": "jwst_plain: " + wp.description + " (one vector per call, forward+gradient)",
                 "l2": "flushed before each step", "roofline_opacity_stage": rl}
        pms, _ = plain_ms(w, w.theta[:1], w.kind[:1])
        plain_same = {"value": 1e3 / pms, "unit": UNIT, "ms_per_spectrum": pms,
                      "workload": args.workload + ": " + w.description +
                      " (one vector per call, forward+gradient)", "l2": "flushed before each step"}

    extra, extra_out, roof_emis = None, {}, None
    if rank == 0 and not args.no_extra:
        extra = []
        for n in ("batched_emis", "highres", "browndwarf", "cloudy_trans", "cloudy_emis", "scattering_emis"):
            want = list(range(8)) if (n in ("batched_emis", "highres") and not args.no_cpu) else None
            rec, wx, gx = measure_workload(n, local, out_vectors=want, probe=(ex2_rate, ffma2_rate), sm_mhz=sm_mhz)
            extra.append(rec)
            if gx is not None:
                extra_out[n] = (wx, gx)
            if n == "batched_emis":
                roof_emis = rec.get("roofline")
        extra.append(measure_nested(local))

    # ---- the FP64 oracle on the host cores (after every GPU timing): the
    # cpu_baseline record, and from the same oracle outputs the BF16-table
    # path's error against the unquantized tables
    cpu, bf16 = None, None
    if rank == 0 and not args.no_cpu:
        pool, cores = oracle_pool()
        try:
            key = (args.workload, args.batch, shard_seed(0))
            cpu, ref = cpu_baseline(pool, cores, key, sample, nfree)
            ref_q = oracle_forwards(pool, key, sample[:4], "bf16") if w.table_dtype == "bf16" else None
            bf16 = {args.workload: bf16_error(gpu_head, ref, ref_q)}
            for n, (wx, gx) in extra_out.items():
                cand = [b for b in valid_vectors(wx, 8) if b in gx["spec"]]
                # one vector of each kind the workload holds, the first with the gradient
                picks = []
                for k in (0, 1):
                    kb = [b for b in cand if int(wx.kind[b]) == k]
                    if kb:
                        picks.append(kb[0])
                keyx = (n, None, 42)
                refx, _ = oracle_gradients(pool, keyx, picks[:1], wx.theta.shape[1])
                refx.update(oracle_forwards(pool, keyx, picks[1:], "fp64"))
                refqx = oracle_forwards(pool, keyx, picks, "bf16")
                gsub = {f: {b: gx[f][b] for b in picks} for f in ("spec", "binned", "lnl")}
                gsub["grad"] = {b: gx["grad"][b] for b in picks[:1]}
                e = bf16_error(gsub, {b: refx[b] for b in picks}, refqx)
                e["kinds"] = [int(wx.kind[b]) for b in picks]
                bf16[n] = e
        finally:
            pool.close()
            pool.join()
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
            "forward_only": forward_only,
            "gpu_launches": int(launches),
            "graph_replay": bool(ctx.es_query(10)),
            "launch_shapes": tuned,
            "ms_per_step_direct_launches": ms_profiled,
            "roofline": roof,
            "roofline_emission": roof_emis,
            "kernels": per_kernel,
            "plain": plain,
            "batched_over_plain": (value / world / plain["value"]) if plain else None,
            "plain_same_workload": plain_same,
            "batched_over_plain_same_workload": (value / world / plain_same["value"]) if plain_same else None,
            "cpu_baseline": cpu,
            "bf16_error": bf16,
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
    """The FP64 oracle as it stands on the host cores (rank 0 only): each step
    is the forward model and complex-step gradient of `REF_VECTORS` parameter
    vectors on whole spectra, one pool task per vector and gradient slot."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2602_19687_gb300 import synth
    key = (args.workload, args.batch, shard_seed(0))
    w = synth.workload(args.workload, batch=args.batch, seed=shard_seed(0))
    nfree = w.theta.shape[1]
    cand = valid_vectors(w, REF_VECTORS * (args.warmup + args.steps))
    pool, cores = oracle_pool()
    per = []
    try:
        for step in range(args.warmup + args.steps):
            vec = [cand[(step * REF_VECTORS + k) % len(cand)] for k in range(REF_VECTORS)]
            _, wall = oracle_gradients(pool, key, vec, nfree)
            per.append(wall)
    finally:
        pool.close()
        pool.join()
    timed = per[args.warmup:]
    sec = float(np.mean(timed))
    sps = REF_VECTORS / sec
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": sps, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded tables, data and parameter batches)",
        "config": {"workload": args.workload + ": " + w.description},
        "cpu_baseline": {"value": sps, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "per step: %d parameter vectors, whole spectra (all %d wavenumbers), forward + "
                                   "complex-step gradient in %d free parameters, FP64 on the unquantized tables, "
                                   "one task per vector and gradient slot over a %d-process pool"
                                   % (REF_VECTORS, w.tables.nu.size, nfree, cores)},
        "e2e": {"value": sps, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def main():
    args = parse()
    if args.oracle_vectors is None:
        args.oracle_vectors = host_cores()
    if args.impl == "reference":
        run_reference(args)
        return
    run_gpu(args)


if __name__ == "__main__":
    main()
