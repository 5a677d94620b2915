"""The spectral shift of the Lanczos operator (the reading that the Lanczos pass runs on
H - tr(H)/D), checked on the CPU with a float32-storage emulation of the pass.

The emulation keeps the vectors in complex64 and forms H.v and the update in float32, as the
mixed-precision path does, takes the dots exactly, and runs the second Gram-Schmidt pass
only on severe cancellation (||w|| < 0.1 ||u||).  On a sparse sector of a long ring the
diagonal offset dominates ||H v||: without the shift the basis loses orthogonality entirely
and beta_j grows far past ||H||; with it the basis stays orthogonal to float rounding and the
tridiagonal matrix keeps the spectrum of H."""
import numpy as np

from oracle import basis as ob
import workloads


def _lanczos_f32(Hc, r0, m, shift):
    f32 = np.complex64
    W, sig, beta = [np.zeros(Hc.D, f32)], [1.0], []
    W[0][r0] = 1
    for j in range(m):
        v = W[j].astype(np.complex128) * sig[j]
        u = (Hc.matvec(v) - shift * v).astype(f32)
        u64 = u.astype(np.complex128)
        c = [np.vdot(W[i].astype(np.complex128) * sig[i], u64) for i in range(j + 1)]
        w = u.copy()
        for i in range(j + 1):
            w = (w - np.complex64(c[i] * sig[i]) * W[i]).astype(f32)
        if np.linalg.norm(w.astype(np.complex128)) < 0.1 * np.linalg.norm(u64):
            c2 = [np.vdot(W[i].astype(np.complex128) * sig[i], w.astype(np.complex128)) for i in range(j + 1)]
            for i in range(j + 1):
                w = (w - np.complex64(c2[i] * sig[i]) * W[i]).astype(f32)
        nw = np.linalg.norm(w.astype(np.complex128))
        beta.append(nw)
        W.append(w)
        sig.append(1.0 / nw)
    V = np.array([W[i].astype(np.complex128) * sig[i] for i in range(m + 1)])
    return np.max(np.abs(V.conj() @ V.T - np.eye(m + 1))), max(beta)


def test_shift_keeps_the_float32_basis_orthogonal():
    L, N = 40, 3
    h = workloads.aubry_andre_field(L, 2.0, 1.0, 0.3, beta=workloads.GOLDEN_Q)
    Hc = ob.CSR(L, N, 1.0, 1.0, h, True)
    r0 = ob.lookup(Hc.basis, (1 << 0) | (1 << 13) | (1 << 26))
    diag = np.array([Hc.val[Hc.rowptr[r]] for r in range(Hc.D)])   # the diagonal is stored first
    norm_bound = Hc.norm_inf()
    orth0, beta0 = _lanczos_f32(Hc, r0, 30, 0.0)
    orth1, beta1 = _lanczos_f32(Hc, r0, 30, float(diag.mean()))
    assert orth0 > 0.1 and beta0 > norm_bound        # unshifted: orthogonality lost
    assert orth1 < 1e-6 and beta1 < norm_bound       # shifted: float-rounding level
