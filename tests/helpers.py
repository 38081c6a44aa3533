"""Comparison helpers shared by the parity tests (no method arithmetic)."""
import numpy as np

# Tolerances: FP64 mode agrees with the FP64 oracle to 1e-12 relative; the
# mixed mode (float32 f, float64 moments) to 1e-5 relative on moments.
TOL_FP64 = 1e-12
TOL_MIXED = 1e-5


def moment_scales(V_ref: np.ndarray) -> np.ndarray:
    """Per-component scale of a conserved field [5, nx]: max|rho|, for the
    momenta max(max|rho u_d|, max rho * sqrt(max theta)) (the thermal momentum,
    so fields that vanish are compared on a physical scale), max|E|."""
    rho = V_ref[0]
    ux, uy, uz = V_ref[1] / rho, V_ref[2] / rho, V_ref[3] / rho
    th = (2 * V_ref[4] / rho - (ux * ux + uy * uy + uz * uz)) / 3
    thermal = np.max(np.abs(rho)) * np.sqrt(np.max(np.abs(th)))
    s = np.empty(5)
    s[0] = np.max(np.abs(V_ref[0]))
    for q in (1, 2, 3):
        s[q] = max(np.max(np.abs(V_ref[q])), thermal)
    s[4] = np.max(np.abs(V_ref[4]))
    return s


def moment_rel_err(V: np.ndarray, V_ref: np.ndarray) -> float:
    """max over components of max|V_q - V_ref_q| / scale_q."""
    s = moment_scales(V_ref)
    return float(np.max(np.max(np.abs(V - V_ref), axis=-1) / s))


def f_rel_err(f: np.ndarray, f_ref: np.ndarray) -> float:
    return float(np.max(np.abs(f - f_ref)) / np.max(np.abs(f_ref)))
