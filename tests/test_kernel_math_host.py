"""The kernels' arithmetic (csrc/fdcgks_math.cuh) compiled for the host and
checked against the oracle without a GPU: interface solves, nodal fluxes and
reconstructions in FP64, and the FP32 erfc of the mixed path to a relative
accuracy of a few FP32 ulp over the whole range, including the tail where erfc
is small (an absolute-error approximation is not enough there)."""
import ctypes
import os
import subprocess

import numpy as np
import pytest
from scipy import special

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2606_17772_gb300", "csrc")
D = ctypes.POINTER(ctypes.c_double)


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("probe") / "libprobe.so")
    subprocess.run(["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-I", CSRC, "-o", out,
                    os.path.join(os.path.dirname(os.path.abspath(__file__)), "host_math_probe.cpp")], check=True)
    return ctypes.CDLL(out)


def _p(a):
    return a.ctypes.data_as(D)


def _states(rng, n, gamma=1.4):
    rho = rng.uniform(0.5, 2.0, n)
    U, V = rng.uniform(-1.5, 1.5, n), rng.uniform(-1.5, 1.5, n)
    p = rng.uniform(0.3, 2.0, n)
    return np.stack([rho, rho * U, rho * V, p / (gamma - 1) + 0.5 * rho * (U * U + V * V)], 1)


@pytest.mark.parametrize("normal", [0, 1])
@pytest.mark.parametrize("mu,Pr,c1,c2", [(0.0, 1.0, 0.05, 1.0), (0.01, 0.73, 0.0, 1.0), (0.0, 1.0, 0.0, 0.0)])
def test_fp64_interface_solve_matches_oracle(probe, normal, mu, Pr, c1, c2):
    rng = np.random.default_rng(3)
    n, dt = 40, 0.004
    Wl = _states(rng, n)
    Wr = Wl * (1 + 0.05 * rng.normal(size=(n, 4)))
    inp = np.ascontiguousarray(np.concatenate([Wl, Wr] + [0.3 * rng.normal(size=(n, 4)) for _ in range(3)], 1))
    out = np.zeros((n, 24))
    probe.probe_iface(0, ctypes.c_double(1.4), ctypes.c_double(mu), ctypes.c_double(Pr), ctypes.c_double(c1),
                      ctypes.c_double(c2), ctypes.c_double(dt), normal, n, _p(inp), _p(out))
    prm = oracle.make_params(8, 8, mu=mu, Pr=Pr, tau_c1=c1, tau_c2=c2)
    ref = np.array([np.concatenate([o[k] for k in ("Fh", "Fht", "Whl", "Whr", "Whlt", "Whrt")]) for o in
                    (oracle.iface_solve(prm, normal, dt, *[inp[t, 4 * k:4 * k + 4] for k in range(5)])
                     for t in range(n))])
    for k in range(6):
        blk = slice(4 * k, 4 * k + 4)
        assert np.abs(out[:, blk] - ref[:, blk]).max() <= 1e-12 * np.abs(ref[:, blk]).max()


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_fp64_reconstruction_matches_oracle(probe, variant):
    rng = np.random.default_rng(variant)
    n, h = 100, 0.1
    Q = 1 + 0.3 * rng.normal(size=(n, 4))
    Qx = 0.5 * rng.normal(size=(n, 4))
    inp = np.ascontiguousarray(np.concatenate([Q, Qx], 1))
    out = np.zeros((n, 6))
    probe.probe_recon(variant, 0, ctypes.c_double(h), n, _p(inp), _p(out))
    ref = np.array([np.concatenate([oracle.recon_left(variant, Q[t], Qx[t, :3], h),
                                    oracle.recon_right(variant, Q[t], Qx[t, 1:], h)]) for t in range(n)])
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12)


def test_fp32_erfc_relative_accuracy(probe):
    """Relative error below 1e-6 from x = -6 to 9 (erfc from 2 down to 4e-37):
    the half-space moments of the kinetic solve need relative accuracy where
    erfc is small, which an absolute bound of 1.5e-7 does not give."""
    x = np.ascontiguousarray(np.linspace(-6.0, 9.0, 6001))
    out = np.zeros_like(x)
    probe.probe_erfc32(len(x), _p(x), _p(out))
    xf = x.astype(np.float32).astype(np.float64)
    ref = special.erfc(xf)
    assert np.max(np.abs(out - ref) / ref) < 1e-6


@pytest.mark.parametrize("variant", [0, 1])
def test_fp32_geno_counts_rounding_level_variation_as_smooth(probe, variant):
    """The FP32 path's rounding floor of the smoothness indicators: lines whose
    values vary by a few FP32 rounding units of their size keep the high-order
    reconstruction (chi = 1), while a genuine jump still turns it off."""
    rng = np.random.default_rng(5 + variant)
    n, h = 200, 0.01
    base = rng.uniform(0.5, 3.0, (n, 1))
    u = np.finfo(np.float32).eps / 2
    Q = np.ascontiguousarray(base * (1 + 4 * u * rng.standard_normal((n, 4))))
    Qx = np.ascontiguousarray(base * 4 * u * rng.standard_normal((n, 4)) / h)
    chi = np.zeros(2 * n)
    probe.probe_recon_chi(1, variant, n, _p(Q), _p(Qx), ctypes.c_double(h), _p(chi))
    assert np.all(chi == 1.0)
    # without the floor (the FP64 path) the same data leave the high-order
    # reconstruction on most lines (252 and 361 of 400 values below 1 measured)
    chi64 = np.zeros(2 * n)
    probe.probe_recon_chi(0, variant, n, _p(Q), _p(Qx), ctypes.c_double(h), _p(chi64))
    assert (chi64 < 1.0).sum() > n
    jump = np.ascontiguousarray(np.tile([1.0, 1.0, 0.125, 0.125], (4, 1)))
    jx = np.zeros_like(jump)
    cj = np.zeros(8)
    probe.probe_recon_chi(1, variant, 4, _p(jump), _p(jx), ctypes.c_double(h), _p(cj))
    assert np.all(cj < 0.5)
    # FP64 has no floor: the same jump gives the same decision
    cd = np.zeros(8)
    probe.probe_recon_chi(0, variant, 4, _p(jump), _p(jx), ctypes.c_double(h), _p(cd))
    assert np.all(cd < 0.5)
