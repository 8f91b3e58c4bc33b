"""The rule that lets the block QR skip its third CholeskyQR pass, restated in numpy on the CPU:
vectors in FP32 (as in the mixed precision), Grams and Cholesky factors in FP64, the product
W R^-1 in FP32 arithmetic.  When the Gram of the second pass's input W R0^-1 is within 1e-2 of the
identity (max entry), one more CholeskyQR pass already leaves the columns orthonormal to the
FP32 level, as a third pass would; for an ill-conditioned W the same test fails, and the third
pass is then what makes the columns orthonormal."""
import numpy as np

f32 = np.float32


def gram(X):
    X64 = X.astype(np.float64)
    return X64.T @ X64


def chol_pass(X, shift=0.0):
    """One CholeskyQR pass: FP64 Gram and factor, the product X R^-1 in FP32 arithmetic."""
    G = gram(X)
    R = np.linalg.cholesky(G + shift * np.trace(G) * np.eye(G.shape[0])).T
    return (X @ np.linalg.inv(R).astype(f32)).astype(f32), G


def orth_err(Q):
    return np.abs(gram(Q) - np.eye(Q.shape[1])).max()


def block(kappa, rows=20000, b=23, seed=0):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((rows, b)))
    V, _ = np.linalg.qr(rng.standard_normal((b, b)))
    s = np.logspace(0, -np.log10(kappa), b)
    return ((U * s) @ V.T).astype(f32)


def three_pass(W, shift):
    W1, _ = chol_pass(W, shift)
    W2, G2 = chol_pass(W1)
    W3, _ = chol_pass(W2)
    return W1, W2, W3, G2


def test_well_conditioned_block_is_orthonormal_after_two_passes():
    for kappa in (1.0, 10.0):
        W1, W2, W3, G2 = three_pass(block(kappa, seed=1), 1e-5)
        dev = np.abs(G2 - np.eye(G2.shape[0])).max()   # the Gram the second pass sees
        assert dev <= 1e-2, (kappa, dev)
        assert orth_err(W2) < 5e-7                       # two passes: orthonormal in FP32
        assert orth_err(W2) < 3 * orth_err(W3)           # as good as three passes


def test_ill_conditioned_block_fails_the_test_and_needs_the_third_pass():
    W1, W2, W3, G2 = three_pass(block(1e5, seed=1), 1e-5)
    dev = np.abs(G2 - np.eye(G2.shape[0])).max()
    assert dev > 1e-2
    assert orth_err(W3) < 5e-7
    assert orth_err(W2) > 10 * orth_err(W3)
