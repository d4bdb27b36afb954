"""C-ABI checks that need no GPU: the library builds and loads, exports every
entry point that include/exoskry.h declares, the ctypes structures match the
C layout, and host-side validation rejects bad arguments before any device
call."""
import ctypes
import os
import re
import subprocess
import tempfile

import numpy as np

import pytest

import __graft_entry__ as entry
from paper_2602_19687_gb300 import binding, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "exoskry.h")


@pytest.fixture(scope="module")
def lib():
    entry.build()
    return binding.load_library()


def header_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:es_status|int64_t|const char \*|void)\s*\**\s*(es_\w+)\(", text, re.M)))


def test_header_declares_the_binding_exports():
    assert header_functions() == sorted(binding.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", binding.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (es_\w+)$", out, re.M))
    for name in header_functions():
        assert name in exported, name
        assert hasattr(lib, name)


def test_struct_layout_matches_c_header():
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "exoskry.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(es_model_desc),
         offsetof(es_model_desc, theta_fixed),
         offsetof(es_model_desc, free_idx), offsetof(es_model_desc, emission_flux),
         offsetof(es_model_desc, distance_cm), offsetof(es_model_desc, cloud_profile),
         offsetof(es_model_desc, cloud_feature), offsetof(es_model_desc, emission_quadrature),
         offsetof(es_model_desc, emission_solver), offsetof(es_model_desc, cloud_ssa),
         offsetof(es_model_desc, cloud_g),
         sizeof(es_tables_desc), offsetof(es_tables_desc, cia_h2he),
         offsetof(es_tables_desc, storage));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    M, T = binding.es_model_desc, binding.es_tables_desc
    assert vals == [ctypes.sizeof(M), M.theta_fixed.offset, M.free_idx.offset, M.emission_flux.offset,
                    M.distance_cm.offset, M.cloud_profile.offset, M.cloud_feature.offset,
                    M.emission_quadrature.offset, M.emission_solver.offset, M.cloud_ssa.offset,
                    M.cloud_g.offset, ctypes.sizeof(T),
                    T.cia_h2he.offset, T.storage.offset]


def test_null_context_calls(lib):
    assert lib.es_query(None, 0) == -1
    assert lib.es_last_error(None) == b"NULL context"
    lib.es_destroy(None)
    assert lib.es_forward(None, None, None, None, 0, None) == binding.ES_EINVAL
    assert lib.es_set_grid(None, None, None, 3) == binding.ES_EINVAL
    assert lib.es_autotune(None, None) == binding.ES_EINVAL
    assert lib.es_set_graphs(None, 1) == binding.ES_EINVAL
    assert lib.es_probe_rates(0, None, None) == binding.ES_EINVAL


@pytest.mark.parametrize("field,value", [("n_layers", 1), ("n_layers", 113), ("n_species", 0),
                                         ("n_species", 17), ("p_top_bar", -1.0), ("tp_kind", 7),
                                         ("cloud_kind", 3), ("n_free", 0), ("r_star_cm", 0.0),
                                         ("emission_flux", 2), ("cloud_profile", 3), ("cloud_profile", -1),
                                         ("cloud_feature", 2), ("emission_quadrature", 2),
                                         ("emission_solver", 2), ("emission_solver", 1)])
def test_create_rejects_bad_descriptions_before_touching_cuda(lib, field, value):
    w = synth.workload("tiny", n_nu=64)
    d = binding.model_desc(w.model)
    setattr(d, field, value)
    h = ctypes.c_void_p()
    assert lib.es_create(ctypes.byref(h), 0, ctypes.byref(d)) == binding.ES_EINVAL
    assert not h.value


@pytest.mark.parametrize("field,value", [("cloud_ssa", -0.1), ("cloud_ssa", 1.5), ("cloud_g", 1.0),
                                         ("cloud_g", -0.2), ("cloud_ssa", float("nan"))])
def test_create_rejects_bad_scattering_constants(lib, field, value):
    """The delta-EAA solver takes a cloud albedo in [0, 1] and an asymmetry
    parameter in [0, 1) (and no grey deck: the tiny workload above)."""
    w = synth.workload("scattering_emis", n_nu=64, batch=1)
    d = binding.model_desc(w.model)
    setattr(d, field, value)
    h = ctypes.c_void_p()
    assert lib.es_create(ctypes.byref(h), 0, ctypes.byref(d)) == binding.ES_EINVAL
    assert not h.value


def test_create_rejects_duplicate_or_out_of_range_free_slots(lib):
    w = synth.workload("tiny", n_nu=64)
    d = binding.model_desc(w.model)
    d.free_idx[1] = d.free_idx[0]
    h = ctypes.c_void_p()
    assert lib.es_create(ctypes.byref(h), 0, ctypes.byref(d)) == binding.ES_EINVAL
    d = binding.model_desc(w.model)
    d.free_idx[0] = 99
    assert lib.es_create(ctypes.byref(h), 0, ctypes.byref(d)) == binding.ES_EINVAL


def test_binding_refuses_to_run_without_the_library(tmp_path):
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        binding._lib = None
        try:
            binding.load_library(str(tmp_path / "missing.so"))
        finally:
            binding._lib = None


def test_host_flux_quadratures_match_the_oracle_rules():
    """The library's host-side angle rules (csrc/quadrature.h: closed-form
    Gauss-Legendre, Golub-Welsch Gauss-Jacobi of the weight mu) against the
    oracle's (numpy leggauss, scipy roots_jacobi), for 4 and 8 points."""
    from oracle import exoskry_oracle as O
    src = r'''
#include <cstdio>
#include "quadrature.h"
int main() {
  double mu[8], w[8];
  es::gauss_legendre4_01(mu, w);
  for (int j = 0; j < 4; ++j) std::printf("%.17g %.17g\n", mu[j], w[j]);
  for (int n = 4; n <= 8; n += 4) {
    es::gauss_jacobi_mu_01(n, mu, w);
    for (int j = 0; j < n; ++j) std::printf("%.17g %.17g\n", mu[j], w[j]);
  }
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "quad.cpp")
        exe = os.path.join(d, "quad")
        open(c, "w").write(src)
        subprocess.run(["g++", "-O2", "-I", os.path.join(ROOT, "paper_2602_19687_gb300", "csrc"), c, "-o", exe],
                       check=True)
        v = np.array([[float(x) for x in line.split()] for line in
                      subprocess.run([exe], capture_output=True, text=True, check=True).stdout.splitlines()])
    mu, w = O.gauss_legendre_01(4)
    np.testing.assert_allclose(v[:4, 0], mu, rtol=0, atol=1e-15)
    np.testing.assert_allclose(v[:4, 1], w, rtol=0, atol=1e-15)
    for n, rows in ((4, slice(4, 8)), (8, slice(8, 16))):
        mu, w = O.gauss_jacobi_mu_01(n)
        np.testing.assert_allclose(v[rows, 0], mu, rtol=0, atol=1e-14)
        np.testing.assert_allclose(v[rows, 1], w, rtol=0, atol=1e-14)


def test_host_mean_intensity_weights_match_the_oracle():
    """The delta-EAA's weights of int_0^1 dmu at the flux angles, as the
    library computes them on the host (csrc/quadrature.h interp_weights_01,
    Gaussian elimination), against the oracle's (numpy solve) at the
    Gauss-Legendre and Gauss-Jacobi nodes, and against the closed forms
    int_0^1 mu^k dmu = 1/(k+1) they integrate exactly."""
    from oracle import exoskry_oracle as O
    src = r'''
#include <cstdio>
#include "quadrature.h"
int main() {
  double mu[8], w[8], c[8];
  es::gauss_legendre4_01(mu, w);
  es::interp_weights_01(4, mu, c);
  for (int j = 0; j < 4; ++j) std::printf("%.17g %.17g\n", mu[j], c[j]);
  es::gauss_jacobi_mu_01(4, mu, w);
  es::interp_weights_01(4, mu, c);
  for (int j = 0; j < 4; ++j) std::printf("%.17g %.17g\n", mu[j], c[j]);
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        cpp = os.path.join(d, "w.cpp")
        exe = os.path.join(d, "w")
        open(cpp, "w").write(src)
        subprocess.run(["g++", "-O2", "-I", os.path.join(ROOT, "paper_2602_19687_gb300", "csrc"), cpp, "-o", exe],
                       check=True)
        v = np.array([[float(x) for x in line.split()] for line in
                      subprocess.run([exe], capture_output=True, text=True, check=True).stdout.splitlines()])
    for rows, kind in ((slice(0, 4), O.QUAD_GAUSS_LEGENDRE), (slice(4, 8), O.QUAD_GAUSS_JACOBI)):
        mu, c = v[rows, 0], v[rows, 1]
        np.testing.assert_allclose(c, O.mean_intensity_weights(O.flux_quadrature(kind, 4)[0]), rtol=0, atol=1e-14)
        for k in range(4):
            assert np.sum(c * mu ** k) == pytest.approx(1.0 / (k + 1), rel=1e-13)
    # at the Gauss-Legendre nodes they are the Gauss-Legendre weights
    np.testing.assert_allclose(v[:4, 1], O.gauss_legendre_01(4)[1], rtol=0, atol=1e-14)


def test_parameter_slots_agree_across_header_binding_synth_and_oracle():
    """The canonical parameter slots (include/exoskry.h ES_P_*) in the same order
    and number in the binding, the synthetic-input module and the oracle."""
    from oracle import exoskry_oracle as O
    src = open(os.path.join(ROOT, "include", "exoskry.h")).read()
    m = re.search(r"enum \{\s*(ES_P_T_ISO = 0,.*?ES_P_N_EXTRA)\s*\};", src, re.S)
    names = [x.strip().split("=")[0].strip()[len("ES_P_"):] for x in m.group(1).split(",")]
    assert names[-1] == "N_EXTRA"
    slots = names[:-1]
    assert len(slots) == binding.ES_P_N_EXTRA == synth.N_EXTRA
    # header name -> the Python modules' name where they differ
    alias = {"LOG_KAPPA_IR": "LOG_KAPPA", "LOG_GAMMA_V": "LOG_GAMMA", "LOG_P_T": "LOG_PT",
             "LOG_P_CLOUD": "LOG_PCLOUD"}
    for k, name in enumerate(slots):
        py = "P_" + alias.get(name, name)
        assert getattr(synth, py) == k, name
        assert getattr(O, py) == k, name
