"""Independent numpy geometry used by the oracle pins (not the oracle, not the CUDA path).

Everything here is written from textbook definitions in a form different from the
oracle's C code, so that agreement between the two pins both."""
import numpy as np


def skew(a):
    a = np.asarray(a, dtype=np.float64)
    return np.array([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]])


def so3_exp(phi):
    """Rodrigues' formula."""
    phi = np.asarray(phi, dtype=np.float64)
    th = np.linalg.norm(phi)
    K = skew(phi)
    if th < 1e-12:
        return np.eye(3) + K + 0.5 * K @ K
    return np.eye(3) + np.sin(th) / th * K + (1 - np.cos(th)) / th ** 2 * K @ K


def se3_exp(xi):
    """exp of xi = (rho, phi) -> (R, t) with t = V rho."""
    rho, phi = np.asarray(xi[:3], float), np.asarray(xi[3:], float)
    th = np.linalg.norm(phi)
    K = skew(phi)
    R = so3_exp(phi)
    if th < 1e-12:
        V = np.eye(3) + 0.5 * K
    else:
        V = np.eye(3) + (1 - np.cos(th)) / th ** 2 * K + (th - np.sin(th)) / th ** 3 * K @ K
    return R, V @ rho


def quat_from_R(R):
    """(w, x, y, z) from a rotation matrix via the eigenvector of Bar-Itzhack's K matrix."""
    m = R
    K = np.array([
        [m[0, 0] - m[1, 1] - m[2, 2], m[1, 0] + m[0, 1], m[2, 0] + m[0, 2], m[2, 1] - m[1, 2]],
        [m[1, 0] + m[0, 1], m[1, 1] - m[0, 0] - m[2, 2], m[2, 1] + m[1, 2], m[0, 2] - m[2, 0]],
        [m[2, 0] + m[0, 2], m[2, 1] + m[1, 2], m[2, 2] - m[0, 0] - m[1, 1], m[1, 0] - m[0, 1]],
        [m[2, 1] - m[1, 2], m[0, 2] - m[2, 0], m[1, 0] - m[0, 1], m[0, 0] + m[1, 1] + m[2, 2]],
    ]) / 3.0
    w, V = np.linalg.eigh(K)
    q = V[:, np.argmax(w)]
    q = np.array([q[3], q[0], q[1], q[2]])
    return q if q[0] >= 0 else -q


def R_from_quat(q):
    """Rotation matrix of a quaternion, via the Hamilton product acting on pure quaternions."""
    q = np.asarray(q, float) / np.linalg.norm(q)

    def mul(a, b):
        w1, x1, y1, z1 = a
        w2, x2, y2, z2 = b
        return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                         w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                         w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                         w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])

    qc = q * np.array([1, -1, -1, -1])
    cols = []
    for e in np.eye(3):
        v = mul(mul(q, np.concatenate([[0.0], e])), qc)
        cols.append(v[1:])
    return np.stack(cols, axis=1)


def bearing(R, t, p):
    pc = R.T @ (np.asarray(p, float) - t)
    return pc / np.linalg.norm(pc)


def landmark_info_closed_form(u, n):
    """6x6 information of one bearing, rotation about the observer, sigma = 1:
    [[P/n^2, -[u]x/n], [[u]x/n, P]] with P = I - u u^T (derived by hand from J^T J)."""
    P = np.eye(3) - np.outer(u, u)
    S = skew(u)
    return np.block([[P / n ** 2, -S / n], [S / n, P]])


def M_shift(a):
    """[[I, -[a]x], [0, I]] : moves the rotation reference point of a 6x6 information by a."""
    M = np.eye(6)
    M[:3, 3:] = -skew(a)
    return M


def Ad(R, t):
    A = np.zeros((6, 6))
    A[:3, :3] = R
    A[:3, 3:] = skew(t) @ R
    A[3:, 3:] = R
    return A


def shell_f32(p, x, r_min, r_max):
    """Range-shell decision in single precision, one rounding per operation (numpy float32)."""
    p = np.asarray(p, np.float32)
    x = np.asarray(x, np.float32)
    d = p - x
    sq = d * d
    n2 = (sq[..., 0] + sq[..., 1]) + sq[..., 2]
    return (n2 > np.float32(r_min * r_min)) & (n2 <= np.float32(r_max * r_max))
