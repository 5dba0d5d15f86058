"""Closed form of the affinely deformed FCC crystal used by the planar
elongational pins (oracle and GPU): a perfect crystal at rest stays a
perfect crystal under grad u = diag(eps, 0, -eps), every site is an
inversion centre (zero force), and the configurational pressure tensor and
energy are sums over one site's neighbour shell."""
import itertools

import numpy as np

RC = 2.0 ** (1.0 / 6.0)


def fcc_vectors(a, reach):
    """FCC lattice vectors (a/2)(n1, n2, n3), n1 + n2 + n3 even, nonzero,
    with every component below `reach` in magnitude."""
    m = int(np.ceil(2 * reach / a)) + 1
    out = []
    for n in itertools.product(range(-m, m + 1), repeat=3):
        if n != (0, 0, 0) and sum(n) % 2 == 0:
            v = 0.5 * a * np.array(n, dtype=float)
            if np.all(np.abs(v) < reach):
                out.append(v)
    return np.array(out)


def lattice_sums(R0, N, V, t, eps):
    """B = P_xx - P_zz and U of the perfect lattice deformed by
    diag(e^{eps t}, 1, e^{-eps t}) with zero momenta:
    W_ab = (N/2) sum_R R_a R_b f(|R|)/|R|, U = (N/2) sum_R phi(|R|)."""
    E = np.array([np.exp(eps * t), 1.0, np.exp(-eps * t)])
    R = R0 * E
    r2 = np.sum(R * R, axis=1)
    R, r2 = R[r2 < RC * RC], r2[r2 < RC * RC]
    s3 = r2 ** -3
    f_over_r = (48.0 * s3 * s3 - 24.0 * s3) / r2
    U = 0.5 * N * np.sum(4.0 * (s3 * s3 - s3) + 1.0)
    B = 0.5 * N * np.sum(f_over_r * (R[:, 0] ** 2 - R[:, 2] ** 2)) / V
    return B, U
