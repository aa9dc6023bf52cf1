"""The hand-written reverse passes of the adjoint (csrc/fdcgks_reverse.cuh)
against forward-mode dual numbers on the same device arithmetic, on the host.

For random inputs and random output adjoints ob, the reverse pass returns
J^T ob; the dual numbers give every Jacobian column J e_i, so (J^T ob)_i =
<ob, J e_i> is checked input by input.  Covered: the kinetic interface solve
for both normals, with and without the first-stage outputs, for viscous,
inviscid, and collision-free (tau = 0) gases and strong jumps; the GENO
interface and node reconstructions for all three constant sets, smooth and
rough data, exact ties of the smoothness indicators; one line with the
positivity safeguard acting on either side; the nodal flux.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2606_17772_gb300", "csrc")
HERE = os.path.dirname(os.path.abspath(__file__))
D = ctypes.POINTER(ctypes.c_double)
GAMMA = 1.4


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("adjprobe") / "libadjprobe.so")
    subprocess.run(["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-I", CSRC, "-I", HERE, "-o", out,
                    os.path.join(HERE, "adjoint_probe.cpp")], check=True)
    return ctypes.CDLL(out)


def _p(a):
    return a.ctypes.data_as(D)


def _state(rng):
    rho, u, v, p = rng.uniform(0.5, 2), rng.uniform(-1.5, 1.5), rng.uniform(-1.5, 1.5), rng.uniform(0.3, 2)
    return np.array([rho, rho * u, rho * v, p / (GAMMA - 1) + 0.5 * rho * (u * u + v * v)])


def _close(rev, dual, tol):
    scale = max(np.abs(dual).max(), 1e-300)
    assert np.abs(rev - dual).max() <= tol * scale, (rev, dual)


GASES = [(0.0, 1.0, 0.05, 1.0), (0.01, 0.73, 0.0, 1.0), (0.0, 1.0, 0.0, 0.0), (0.5, 0.72, 0.0, 1.0)]


@pytest.mark.parametrize("gas", range(len(GASES)))
def test_solve_reverse_equals_dual_numbers(probe, gas):
    mu, Pr, c1, c2 = GASES[gas]
    rng = np.random.default_rng(gas)
    for t in range(30):
        Wl = _state(rng)
        Wr = Wl * (1 + 0.05 * rng.normal(size=4)) if t % 3 else _state(rng)    # strong jumps too
        if t == 0:
            Wr = Wl.copy()                                                      # |p_l - p_r| = 0
        inp = np.concatenate([Wl, Wr] + [0.3 * rng.normal(size=4) for _ in range(3)])
        ob = rng.normal(size=24)
        for normal in (0, 1):
            for wn in (0, 1):
                rev, dual = np.zeros(20), np.zeros(20)
                probe.probe_solve_vjp(ctypes.c_double(GAMMA), ctypes.c_double(mu), ctypes.c_double(Pr),
                                      ctypes.c_double(c1), ctypes.c_double(c2), ctypes.c_double(0.004), normal, wn,
                                      _p(inp), _p(ob), _p(rev), _p(dual))
                _close(rev, dual, 1e-11)


def _lines(rng, n):
    rows = []
    for t in range(n):
        kind = t % 4
        if kind == 0:
            Q = 1 + np.cumsum(0.02 * rng.normal(size=4))             # smooth
        elif kind == 1:
            Q = 1 + 0.3 * rng.normal(size=4)                          # rough
        elif kind == 2:
            Q = np.full(4, 1.3)                                       # constant: every IS_k = 0 (ties)
        else:
            x = np.arange(4.0)
            Q = 0.7 + 0.1 * x + 0.02 * x * x                          # quadratic: equal IS_k
        Qx = 0.5 * rng.normal(size=4) if kind < 2 else np.zeros(4)
        rows.append((Q, Qx))
    return rows


FLOOR = 64 * 2.0 ** -24          # the FP32 path's floor scale, for the reverse pass of a mixed run


@pytest.mark.parametrize("fscale", [0.0, FLOOR])
@pytest.mark.parametrize("variant", [0, 1, 2])
def test_reconstruction_reverse_equals_dual_numbers(probe, variant, fscale):
    """fscale > 0: the path function with the FP32 path's rounding floor
    (64 u max|Q|)^2 added to eps_a, evaluated in FP64, including the floor's
    own dependence on the data."""
    rng = np.random.default_rng(10 + variant)
    rows = _lines(rng, 200)
    # data varying by about the floor: there the floor decides chi
    for t in range(40):
        rows.append((1.0 + 3e-6 * rng.normal(size=4), 3e-5 * rng.normal(size=4)))
    for Q, Qx in rows:
        inp = np.concatenate([Q, Qx])
        ob = rng.normal(size=6)
        rev, dual = np.zeros(8), np.zeros(8)
        probe.probe_recon_iface_vjp(variant, ctypes.c_double(0.07), ctypes.c_double(fscale), _p(inp), _p(ob),
                                    _p(rev), _p(dual))
        _close(rev, dual, 1e-11)
        inp3 = np.concatenate([Q[:3], Qx[:3]])
        rev, dual = np.zeros(6), np.zeros(6)
        probe.probe_recon_node_vjp(variant, ctypes.c_double(0.07), ctypes.c_double(fscale), _p(inp3),
                                   ctypes.c_double(ob[0]), _p(rev), _p(dual))
        _close(rev, dual, 1e-11)


@pytest.mark.parametrize("fscale", [0.0, FLOOR])
@pytest.mark.parametrize("variant", [0, 1])
def test_line_reverse_with_positivity_safeguard(probe, variant, fscale):
    """Lines whose reconstructed left or right state has negative pressure
    (the safeguard replaces it by the node state) and ordinary lines."""
    rng = np.random.default_rng(20 + variant)
    acted = 0
    for t in range(60):
        W = np.array([_state(rng) for _ in range(4)])
        if t % 2 == 0:
            # a strong jump with a low-pressure side: reconstructions overshoot
            W[2:] = W[2:] * np.array([0.01, 0.001, 0.001, 0.0005])
        G = 20.0 * rng.normal(size=(4, 4)) * np.abs(W)
        x = np.concatenate([np.concatenate([W[e], G[e]]) for e in range(4)])
        ob = rng.normal(size=17)
        rev, dual = np.zeros(32), np.zeros(32)
        flag = ctypes.c_int()
        probe.probe_recon_line_vjp(variant, ctypes.c_double(0.05), ctypes.c_double(fscale), _p(x), _p(ob), _p(rev),
                                   _p(dual), ctypes.byref(flag))
        _close(rev, dual, 1e-11)
        acted |= flag.value
    assert acted == 3          # the safeguard acted on left and on right states


def test_nodal_flux_reverse_equals_dual_numbers(probe):
    rng = np.random.default_rng(30)
    for mu, Pr, c1 in ((0.0, 1.0, 0.05), (0.01, 0.73, 0.0), (0.5, 0.72, 0.0)):
        for _ in range(30):
            inp = np.concatenate([_state(rng), 0.3 * rng.normal(size=8)])
            ob = rng.normal(size=16)
            rev, dual = np.zeros(12), np.zeros(12)
            probe.probe_nodal_vjp(ctypes.c_double(GAMMA), ctypes.c_double(mu), ctypes.c_double(Pr),
                                  ctypes.c_double(c1), ctypes.c_double(0.004), _p(inp), _p(ob), _p(rev), _p(dual))
            _close(rev, dual, 1e-11)
