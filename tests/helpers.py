"""Shared helpers for the GPU parity tests: run the CUDA path (through the C
ABI) and the oracle on the same seeded case and collect comparable states."""
import numpy as np

from oracle.gsis import OracleSolver

# FP64 tolerance on macroscopic fields (relative), the stated target of the path.
RTOL_W = 1e-10


def rel_err(a, b, scale=None):
    a = np.asarray(a); b = np.asarray(b)
    s = np.max(np.abs(b)) if scale is None else scale
    return float(np.max(np.abs(a - b)) / max(s, 1e-300))


def w_rel_err(Wg, Wo):
    """Max over the five primitive fields of max|dW| / max|W| (velocity as one field)."""
    errs = [rel_err(Wg[:, 0], Wo[:, 0]), rel_err(Wg[:, 1:4], Wo[:, 1:4]), rel_err(Wg[:, 4], Wo[:, 4])]
    return max(errs)


def run_oracle(case, n_iter, flags=None):
    o = OracleSolver(case, flags_override=flags)
    o.initialise()
    hist = [o.W.copy()]
    for _ in range(n_iter):
        o.step()
        hist.append(o.W.copy())
    return o, hist


def run_gpu(case, n_iter, vdf_dtype="f64", flags=None):
    from paper_2501_02245_gb300 import Solver
    s = Solver.from_case(case, vdf_dtype=vdf_dtype, forced_flags=flags)
    s.iterate(0)
    hist = [s.W()]
    reps = []
    for _ in range(n_iter):
        reps.append(s.iterate(1))
        hist.append(s.W())
    return s, hist, reps


def vdf_by_cell(solver, n_dvm, ncell, nv):
    cells, f = solver.vdf(n_dvm)
    full = np.zeros((ncell, nv))
    full[cells] = f
    return full


def moment_scales(direct):
    """Per-component magnitude of each moment order of gsis_debug_vdf_moments
    over all cells: rho, rho sqrt(T), rho T, rho T^(3/2) (from the direct
    moments), and the largest wall sum."""
    s0 = np.abs(direct[:, 0]).max()
    s2 = np.abs(direct[:, 4] + direct[:, 5] + direct[:, 6]).max() / 3.0
    s1 = np.sqrt(s0 * s2)
    s3 = s2 ** 1.5 / np.sqrt(s0)
    sw = max(np.abs(direct[:, 13:]).max(), 1e-300)
    return np.array([s0] + [s1] * 3 + [s2] * 6 + [s3] * 3 + [sw] * 6)


def compare_derived(s, o, tol):
    """Wall pressure and shear, the constitutive stress and heat flux of Eq.
    full_constitutive at the current state, and the pressure."""
    names = ["wall_p", "wall_tx", "wall_ty", "wall_tz", "sxx", "syy", "szz", "sxy", "sxz", "syz",
             "qx", "qy", "qz", "p"]
    g = s.moments(names)
    L = o.wall_loads()
    if np.any(L[:, 1] != 0.0):
        assert rel_err(g["wall_p"], L[:, 1]) < tol
        tau = np.stack([g["wall_tx"], g["wall_ty"], g["wall_tz"]], axis=1)
        assert rel_err(tau, L[:, 2:5]) < tol, "wall shear relative error %.3e" % rel_err(tau, L[:, 2:5])
    sig_o, q_o = o.constitutive()
    sig = np.stack([g[k] for k in ("sxx", "syy", "szz", "sxy", "sxz", "syz")], axis=1)
    e = rel_err(sig, sig_o[:, [0, 1, 2, 0, 0, 1], [0, 1, 2, 1, 2, 2]])
    assert e < tol, "constitutive stress relative error %.3e" % e
    q = np.stack([g[k] for k in ("qx", "qy", "qz")], axis=1)
    assert rel_err(q, q_o) < tol, "constitutive heat flux relative error %.3e" % rel_err(q, q_o)
    assert rel_err(g["p"], o.W[:, 0] * o.W[:, 4]) < 1e-12
