"""Layout conversions between the oracle (class-major, separate blocks) and the C ABI
(pixel-major state arrays), and the seeded cases shared by the GPU tests."""
import numpy as np

from oracle import segsalsa_str_oracle as O


def khw_to_hwk(a):
    return np.ascontiguousarray(np.moveaxis(a, 0, -1))


def hwk_to_khw(a):
    return np.ascontiguousarray(np.moveaxis(a, -1, 0))


def d2_oracle_to_abi(d2):
    """(L, K, 2, H, W) -> (H, W, L, K, 2)."""
    return np.ascontiguousarray(np.transpose(d2, (3, 4, 0, 1, 2)))


def d2_abi_to_oracle(d2):
    return np.ascontiguousarray(np.transpose(d2, (2, 3, 4, 0, 1)))


def oracle_state_to_abi(st: O.SalsaState, omega, M, dtype):
    """Checkpoint arrays of the C ABI for an oracle state after st.k iterations."""
    out = {
        "z": khw_to_hwk(st.z),
        "d1": khw_to_hwk(st.d[0]),
        "d2": d2_oracle_to_abi(st.d[1]),
        "d3": khw_to_hwk(st.d[2]),
        "d4": khw_to_hwk(st.d[3]),
        "rhs": khw_to_hwk(st.rhs(omega, M)) if st.k > 0 else None,
    }
    return {k: (None if v is None else v.astype(dtype)) for k, v in out.items()}


def max_abs(a, b):
    return float(np.max(np.abs(np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64))))


def label_agreement(z_gpu_khw, z_ref_khw, margin_tol=1e-3):
    """Labels must agree except where the reference top-two margin is below margin_tol."""
    lab_g = np.argmax(z_gpu_khw, axis=0)
    lab_r, margin = O.labels_and_margin(z_ref_khw)
    clear = margin >= margin_tol
    return bool(np.all(lab_g[clear] == lab_r[clear])), int(np.sum(~clear))
