"""The dense FP64 eigensolver of the Rayleigh-Ritz step (qm_eigh_lowest through the C ABI)
against LAPACK's eigvalsh on seeded Hermitian matrices: eigenvalues to 1e-12 |A|,
eigen-residuals to 1e-12 |A|, orthonormality to 1e-10 (inverse iteration outside clusters
leaves eps |T| / gap), including exactly degenerate clusters, a long chain of close eigenvalues
and already-diagonal input."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2308_07277_gb300 as Q
    return Q


def _herm(rng, m):
    X = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    return 0.5 * (X + X.conj().T)


def _check(Q, H, nev):
    ev, Y = Q.qm_eigh_lowest(torch.from_numpy(H).cuda(), nev)
    torch.cuda.synchronize()
    ev, Y = ev.cpu().numpy(), Y.cpu().numpy()
    full = np.linalg.eigvalsh(H)
    ref = full[:nev]
    scale = max(1.0, np.abs(full).max())
    assert np.abs(ev - ref).max() <= 1e-12 * scale
    assert np.abs(H @ Y - Y * ev).max() <= 1e-12 * scale
    assert np.abs(Y.conj().T @ Y - np.eye(nev)).max() <= 1e-10


# sizes span the three reduction kernels: rows in shared memory (m <= ~1100), rows updated in
# place in device memory (m = 1216), and the two-barrier kernel (m = 3240)
@pytest.mark.parametrize("m,nev", [(1, 1), (2, 1), (3, 2), (7, 7), (64, 20), (333, 111), (640, 160), (704, 176),
                                   (960, 480), (1216, 100), (3240, 12)])
def test_random_hermitian(Q, m, nev):
    _check(Q, _herm(np.random.default_rng(m), m), nev)


def test_degenerate_clusters(Q):
    rng = np.random.default_rng(5)
    B = _herm(rng, 40)
    H = np.kron(np.eye(3), B)                              # every eigenvalue 3-fold
    U, _ = np.linalg.qr(rng.standard_normal((120, 120)) + 1j * rng.standard_normal((120, 120)))
    H = U @ H @ U.conj().T
    _check(Q, 0.5 * (H + H.conj().T), 30)


def test_diagonal_and_zero_coupling(Q):
    d = np.linspace(-3.0, 5.0, 50)
    _check(Q, np.diag(d).astype(np.complex128), 25)
    H = np.zeros((6, 6), complex)                          # the zero matrix: all eigenvalues 0
    _check(Q, H, 6)


def test_long_cluster_chain(Q):
    """60 eigenvalues 1e-7 apart (one cluster chain for the inverse iteration) among others."""
    rng = np.random.default_rng(11)
    m = 300
    lam = np.concatenate([-1.0 + 1e-7 * np.arange(60), np.linspace(0.5, 4.0, m - 60)])
    U, _ = np.linalg.qr(rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m)))
    H = (U * lam) @ U.conj().T
    _check(Q, 0.5 * (H + H.conj().T), 80)
