"""Host-side checks of the native library that need no GPU: it builds for
sm_103a, loads, exports every symbol that include/odegpu.h declares, and its
pure host helpers agree with the oracle's independent implementations."""
import os
import re
import subprocess

import numpy as np
import pytest

import oracle as O
import workloads as W
from paper_1810_03931_gb300 import build as B
from paper_1810_03931_gb300 import odegpu as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_symbols():
    txt = open(os.path.join(ROOT, "include", "odegpu.h")).read()
    return sorted(set(re.findall(r"^(?:int|const char \*)\s*\**(ode_\w+)\s*\(", txt, re.M)))


def test_library_builds_and_exports_every_declared_symbol():
    lib = B.build()
    assert os.path.exists(lib)
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (ode_\w+)$", out, re.M))
    declared = _header_symbols()
    assert len(declared) >= 20
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    assert set(G.SYMBOLS) == set(declared)
    L = G.load()
    for s in declared:
        assert hasattr(L, s)


def test_kernels_are_compiled_for_sm_103a():
    objdir = B.BUILD
    assert any(f.startswith("kern_") for f in os.listdir(objdir))
    assert any(f == "-gencode" for f in B.NVCC_FLAGS)
    assert "arch=compute_103a,code=sm_103a" in B.NVCC_FLAGS


def test_create_without_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(G.ODEError) as e:
        G.ode_create(G.ODE_DUFFING, G.ODE_RKCK45, G.ODE_FP64, 16, 0)
    assert e.value.code in (G.ODE_ERR_CUDA, G.ODE_ERR_INVALID_ARG)
    assert G.ode_last_error()


def test_argument_validation_before_any_device_work():
    with pytest.raises(G.ODEError) as e:
        G.ode_create(9, 0, 0, 16, 0)
    assert e.value.code == G.ODE_ERR_INVALID_ARG
    with pytest.raises(G.ODEError) as e:
        G.ode_create(G.ODE_KELLER_MIKSIS, 1, G.ODE_FP32_RHS, 16, 0)
    assert e.value.code == G.ODE_ERR_INVALID_ARG
    with pytest.raises(G.ODEError) as e:
        G.ode_create(G.ODE_DUFFING, 1, 0, 0, 0)
    assert e.value.code == G.ODE_ERR_INVALID_ARG


def test_km_coefficients_agree_with_the_oracle():
    """Two independent codings of Eqs. (16)-(28)."""
    w = W.keller_miksis(7, 5, 0, 1)
    ph = w["phys"]
    ref = O.km_coefficients(w["PA"], w["omega"], PA2=0.3e5, omega2=2 * w["omega"], theta=0.4, **ph)
    for i in range(w["N"]):
        c = G.ode_km_coefficients(w["PA"][i], 0.3e5, w["omega"][i], 2 * w["omega"][i], 0.4, ph["RE"],
                                  ph["Pinf"], ph["pV"], ph["sigma"], ph["mu"], ph["rho"], ph["cL"],
                                  ph["gamma"])
        np.testing.assert_allclose(c, ref[:, i], rtol=1e-14, atol=0)


def test_workload_generators_are_seeded_and_shaped():
    a = W.duffing_rkck()
    assert a["N"] == 2 ** 17 and a["p"].shape == (2, 2 ** 17)
    assert a["p"][0, 1] > a["p"][0, 0] and a["p"][1, 511] == a["p"][1, 0]  # k fastest
    k = W.keller_miksis()
    assert k["N"] == 2 ** 18
    v = W.valve()
    assert v["N"] == 2 ** 16 and v["p"][3, 0] == 0.2 and v["p"][3, -1] == 10.0
    s1, s2 = W.serving_mix(50), W.serving_mix(50)
    assert s1 == s2
    assert all(1 <= r["size"] <= 2 ** 16 and 16 <= r["horizon"] <= 1024 for r in s1)
    idx = W.sample_indices(1000, 20, corners=(0, 999))
    assert len(idx) == 20 and 0 in idx and 999 in idx


def _morton_reference(keys):
    """Z-order of the columns of `keys` written independently: each key
    scaled to [0, 1] over its range, quantized to b = min(31, 63 // K) bits,
    codes compared as bit strings interleaved most significant first."""
    K, N = keys.shape
    b = min(31, 63 // K)
    q = np.zeros((K, N), dtype=np.int64)
    for d in range(K):
        lo, hi = keys[d].min(), keys[d].max()
        if hi > lo:
            q[d] = np.floor((keys[d] - lo) / (hi - lo) * (2 ** b - 1) + 0.5).astype(np.int64)
    def code(i):
        return tuple((int(q[d, i]) >> bit) & 1 for bit in reversed(range(b)) for d in reversed(range(K)))
    return sorted(range(N), key=lambda i: (code(i), i))


def test_cluster_order_is_a_z_order_permutation():
    rng = np.random.default_rng(7)
    for K, N in ((1, 50), (2, 300), (3, 200)):
        keys = rng.random((K, N))
        keys[0, :5] = keys[0, 5]  # ties keep index order
        perm = G.ode_cluster_order(keys)
        assert list(perm) == _morton_reference(keys)
    # a constant key orders nothing; non-finite keys go last
    k = np.vstack([np.linspace(0, 1, 8)[::-1], np.full(8, 3.0)])
    assert list(G.ode_cluster_order(k)) == list(range(8))[::-1]
    k = np.array([[0.5, np.nan, 0.1, np.inf, 0.9]])
    assert list(G.ode_cluster_order(k)) == [2, 0, 4, 1, 3]
    # neighbours in the order are close in parameter space
    g = np.stack(np.meshgrid(np.linspace(0, 1, 32), np.linspace(0, 1, 32))).reshape(2, -1)
    sh = g[:, rng.permutation(g.shape[1])]
    cl = sh[:, G.ode_cluster_order(sh)]
    step = lambda a: np.mean(np.abs(np.diff(a, axis=1)).sum(axis=0))
    assert step(cl) < 0.1 * step(sh)
    with pytest.raises(G.ODEError):
        G.ode_cluster_order(np.zeros((9, 4)))


def test_bench_uses_a_measured_traffic_only_for_its_kernel_sources(tmp_path):
    import json
    import sys
    sys.path.insert(0, ROOT)
    import bench
    path = str(tmp_path / "t.json")
    entry = {"per_sweep": {"source_sha256": bench.kernel_source_digest(), "dram_bytes_per_launch": 1.5e9}}
    json.dump({"duffing_rkck_512x256": entry}, open(path, "w"))
    assert bench.measured_traffic("duffing_rkck_512x256", 0, path) == 1.5e9
    assert bench.measured_traffic("duffing_rkck_512x256", 1, path) is None  # other launch form
    assert bench.measured_traffic("valve_65536", 0, path) is None
    entry["per_sweep"]["source_sha256"] = "0" * 64  # taken on other sources
    json.dump({"duffing_rkck_512x256": entry}, open(path, "w"))
    assert bench.measured_traffic("duffing_rkck_512x256", 0, path) is None
