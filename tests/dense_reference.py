"""Dense Kronecker-product construction of the Floquet operator (L <= 10).

Used only to pin the oracle: every operator here is built from Pauli strings
with numpy.kron and exponentiated with scipy.linalg.expm, independently of the
oracle's index pairing and of its Taylor exponential.  Site i is bit i of the
amplitude index, so the Kronecker order is (site L-1) x ... x (site 0).
"""
import numpy as np
import scipy.linalg as sla

I2 = np.eye(2, dtype=np.complex128)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)


def site_op(L, i, A):
    out = np.array([[1.0 + 0j]])
    for s in range(L - 1, -1, -1):
        out = np.kron(out, A if s == i else I2)
    return out


def two_site_op(L, i, M):
    """Embed a 4x4 operator whose local index is r = 2 b_i + b_{i+1}."""
    dim = 1 << L
    out = np.zeros((dim, dim), dtype=np.complex128)
    mask = (1 << i) | (1 << (i + 1))
    for xo in range(dim):
        ro = 2 * ((xo >> i) & 1) + ((xo >> (i + 1)) & 1)
        for ri in range(4):
            xi = (xo & ~mask) | (((ri >> 1) & 1) << i) | ((ri & 1) << (i + 1))
            out[xo, xi] += M[ro, ri]
    return out


def ising_bond_dense(L, b, J, hx, hz, ew):
    wl = ew if b == 0 else 0.5
    wr = ew if b + 1 == L - 1 else 0.5
    i, j = b, b + 1
    return (J * site_op(L, i, Z) @ site_op(L, j, Z)
            + hx * (wl * site_op(L, i, X) + wr * site_op(L, j, X))
            + hz * (wl * site_op(L, i, Z) + wr * site_op(L, j, Z)))


def floquet_dense(bond_terms, L, tau, theta, K, first_layer):
    """U_F = exp(-i theta sum X) (U_second U_first)^K with
    U_parity = expm(-i tau sum_{b in parity} h_b)."""
    dim = 1 << L
    layers = []
    for parity in (first_layer, 1 - first_layer):
        H = np.zeros((dim, dim), dtype=np.complex128)
        for b in range(parity, L - 1, 2):
            H += bond_terms[b]
        layers.append(sla.expm(-1j * tau * H))
    step = layers[1] @ layers[0]
    U = np.linalg.matrix_power(step, K)
    SX = sum(site_op(L, i, X) for i in range(L))
    return sla.expm(-1j * theta * SX) @ U


def product_state_dense(spinors):
    psi = np.array([1.0 + 0j])
    for i in range(spinors.shape[0] - 1, -1, -1):
        v = np.array([spinors[i, 0] + 1j * spinors[i, 1], spinors[i, 2] + 1j * spinors[i, 3]])
        psi = np.kron(psi, v)
    return psi
