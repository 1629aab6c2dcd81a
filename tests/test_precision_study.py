"""Why the mixed-precision path keeps its Lanczos basis V in FP32 rather than
BF16 (a CPU study, numpy + the oracle's Wilson operator; no GPU).

The seed recurrence of Sec. 3 is run with FP32 Krylov vectors and FP64 scalars,
as the mixed-precision GPU path runs it, with periodic reorthogonalization (two
classical Gram-Schmidt passes every 25 steps) against the stored basis V, stored
either in FP32 or rounded to BF16 (round to nearest even; the storage the
paper-independent BF16 option would use).  Workload: 6^4 Wilson lattice,
kappa 0.150, links exp(0.3 i H) from seed 0, b = D^H eta with Z4 noise eta,
seed tolerance 1e-7.

A BF16 basis leaves components of the size of its rounding (2^-9) after each
Gram-Schmidt pass, which the recurrence then amplifies: the stored basis loses
orthogonality and the seed solution's true residual is far worse than with an
FP32 basis.  The numbers are printed by the test (pytest -s).
"""
import numpy as np

from paper_0810_0330_gb300 import inputs as I


def _bf16(x: np.ndarray) -> np.ndarray:
    """Round complex64 entries to BF16 (nearest even) and back to complex64."""
    def r(a):
        b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
        b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
        return b.astype(np.uint32).view(np.float32)
    return (r(x.real) + 1j * r(x.imag)).astype(np.complex64)


def _seed_run(op, b, store, freq=25, tol=1e-7, m_max=400):
    """Sec. 3 seed recurrence on one right-hand side: FP32 vectors (v, f, w, x),
    FP64 scalars, the operator applied in FP64 to the FP32 vector and rounded;
    `store` rounds a vector into the basis V.  Returns (steps, stored V, x)."""
    apply32 = lambda v: op.apply(v.astype(np.complex128)).astype(np.complex64)
    dot = lambda a, c: complex(np.vdot(a.astype(np.complex128), c.astype(np.complex128)))
    bn = np.linalg.norm(b)
    beta0 = bn
    v = (b / beta0).astype(np.complex64)
    V = [store(v)]
    f = apply32(v)
    alpha = dot(v, f).real
    f = (f - np.complex64(alpha) * v).astype(np.complex64)
    delta = alpha
    w = (v / np.float32(delta)).astype(np.complex64)
    zeta = beta0
    x = (np.float32(zeta) * w).astype(np.complex64)
    i = 1
    while True:
        beta = float(np.linalg.norm(f.astype(np.complex128)))
        if beta * abs(zeta) / delta <= tol * bn or i >= m_max:
            break
        v_prev, v = v, (f / np.float32(beta)).astype(np.complex64)
        i += 1
        V.append(store(v))
        f = (apply32(v) - np.float32(beta) * v_prev).astype(np.complex64)
        alpha = dot(v, f).real
        f = (f - np.float32(alpha) * v).astype(np.complex64)
        gamma = beta / delta
        delta = alpha - gamma * beta
        w = ((v - np.float32(beta) * w) / np.float32(delta)).astype(np.complex64)
        zeta = -gamma * zeta
        x = (x + np.float32(zeta) * w).astype(np.complex64)
        if i % freq == 0:
            for tgt, k in (("v", i - 1), ("f", i)):
                y = v if tgt == "v" else f
                B = np.stack(V[:k], axis=1).astype(np.complex128)
                for _ in range(2):       # classical Gram-Schmidt, two passes, FP64 coefficients
                    h = B.conj().T @ y.astype(np.complex128)
                    y = (y.astype(np.complex128) - B @ h).astype(np.complex64)
                if tgt == "v":
                    v = (y / np.float32(np.linalg.norm(y.astype(np.complex128)))).astype(np.complex64)
                    V[i - 1] = store(v)
                else:
                    f = y
    return i, np.stack(V, axis=1), x


def test_bf16_basis_loses_orthogonality_and_accuracy(orc):
    dims, kappa = (6, 6, 6, 6), 0.150
    U = I.random_su3_links(dims, 0.3, seed=0)
    n = 12 * I.lattice_sites(dims)
    eta = I.z4_noise(n, 1, seed=0)[:, 0]
    b = orc.wilson_dslash(dims, kappa, 0, -1, U, eta)
    op = orc.Operator.wilson(dims, kappa, U)
    res = {}
    for name, store in (("fp32", lambda v: v.copy()), ("bf16", _bf16)):
        steps, V, x = _seed_run(op, b, store)
        G = V.astype(np.complex128).conj().T @ V.astype(np.complex128)
        offdiag = np.abs(G - np.diag(np.diag(G))).max()
        relres = np.linalg.norm(b - op.apply(x.astype(np.complex128))) / np.linalg.norm(b)
        res[name] = (steps, offdiag, relres)
        print("%s basis: %d steps, max |V^H V - diag| = %.2e, true relative residual of x^1 = %.2e"
              % (name, steps, offdiag, relres))
    (s32, o32, r32), (s16, o16, r16) = res["fp32"], res["bf16"]
    assert o16 >= 10 * o32, (o16, o32)
    assert r16 >= 5 * r32, (r16, r32)
    assert r32 <= 5e-6
