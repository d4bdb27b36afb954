"""Error of the BF16-table path against the FP64 oracle on the unquantized
tables (the tables as generated, before the library stores each row as BF16
residuals about an FP32 row mean).

The GPU parity tests compare the kernels with the oracle run on the same
BF16-stored table values (the arithmetic's error). Here the reference is the
FP64 model on the original tables, so the measured difference is the whole
error a user of the BF16 storage sees: the quantization of log10 sigma (half
a BF16 ulp of the residual, at most 0.0078 dex for |residual| < 4) carried
through the interpolation, the chord optical depth or the emission integral,
the binning, ln L and the gradient. Measured on the batched transmission and
batched emission workloads at full size and on the high-resolution mixed
batch on a tenth of its wavenumber grid; the bounds asserted are about twice
the quantization error the oracle alone measures on the same vectors.
"""
import numpy as np
import pytest

import bench
from paper_2602_19687_gb300 import binding, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"

# workload, n_nu, vectors, bounds: native spectrum (max relative), binned
# model (max relative), ln L (max relative), gradient (max relative per
# component, floor 1e-3 of the largest). The quantization alone (the FP64
# oracle on the BF16-stored values against it on the original tables, same
# vectors) measured: transmission native 2.1e-4, binned 6.0e-6, ln L 4.1e-7,
# gradient 3.4e-5; emission 1.4e-2, 1.7e-4, 4.9e-6, 2.0e-4; the mixed
# high-resolution batch 3.8e-4, 6.9e-6, 5.4e-7, 2.8e-5. The gradient bound
# also covers the adjoint's own FP32 error (up to ~2e-4 per component).
CASES = [
    ("batched_trans", None, 3, dict(native=5e-4, binned=1.5e-5, lnl=1e-6, grad=2e-3)),
    ("batched_emis", None, 3, dict(native=3e-2, binned=4e-4, lnl=1e-5, grad=2e-3)),
    ("highres", 44000, 3, dict(native=1e-3, binned=2e-5, lnl=2e-6, grad=2e-3)),
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.fixture(scope="module")
def pool():
    p, n = bench.oracle_pool()
    yield p
    p.close()
    p.join()


def _gpu(w, vec):
    ctx = binding.context_for(w)
    B = w.theta.shape[0]
    th = torch.tensor(w.theta, dtype=torch.float64, device=DEV)
    ctx.es_set_batch(th, torch.tensor(w.kind, dtype=torch.int32, device=DEV))
    spec = torch.empty((B, w.tables.nu.size), dtype=torch.float32, device=DEV)
    binned = torch.empty((B, w.bin_lo_um.size), dtype=torch.float64, device=DEV)
    lnl = torch.empty(B, dtype=torch.float64, device=DEV)
    ctx.es_forward(spectrum=spec, binned=binned, lnl=lnl)
    lnl2 = torch.empty_like(lnl)
    grad = torch.empty_like(th)
    ctx.es_forward_backward(lnl2, grad)
    torch.cuda.synchronize()
    ctx.es_destroy()
    return {"spec": {b: spec[b].cpu().numpy().astype(np.float64) for b in vec},
            "binned": {b: binned[b].cpu().numpy() for b in vec},
            "lnl": {b: float(lnl[b]) for b in vec}, "grad": {b: grad[b].cpu().numpy() for b in vec[:1]}}


@pytest.mark.parametrize("name,n_nu,nvec,bound", CASES, ids=[c[0] for c in CASES])
def test_bf16_tables_error_against_fp64(pool, name, n_nu, nvec, bound):
    w = synth.workload(name, batch=8, n_nu=n_nu)
    assert w.table_dtype == "bf16"
    vec = bench.valid_vectors(w, nvec)
    gpu = _gpu(w, vec)
    key = (name, 8, 42, n_nu)
    ref, _ = bench.oracle_gradients(pool, key, vec[:1], w.theta.shape[1])
    ref.update(bench.oracle_forwards(pool, key, vec[1:], "fp64"))
    ref_q = bench.oracle_forwards(pool, key, vec, "bf16")
    e = bench.bf16_error(gpu, ref, ref_q)
    print("\nbf16 error %s: %s" % (name, e))
    assert e["vectors"] == len(vec) and e["grad_vectors"] == 1
    assert e["native"]["max"] < bound["native"]
    assert e["binned"]["max"] < bound["binned"]
    assert e["lnl_rel"]["max"] < bound["lnl"]
    assert e["grad"]["max"] < bound["grad"]
    # the GPU arithmetic on the stored values: the transit-depth parity
    # tolerance for transmission; emission fluxes are compared relative to
    # each point, also where the flux is far below its maximum
    tol = 1e-5 if np.all(w.kind[vec] == 0) else 1e-3
    assert e["gpu_arithmetic_only"]["native"]["max"] < tol
