"""The eigensolver's tall-skinny contractions (the Gram matrices and block updates of the
Rayleigh-Ritz step, Sec. 4.1, Alg. 2 in block form) against their plain definition, a numpy
FP64 matrix product, through the C ABI (iwf_gram, iwf_block_update).

Tolerances follow from the arithmetic. The tensor-core engine rounds every value once to a
56-bit fixed-point integer under its group's power-of-two scale (|error| <= 2^-56 of the
scale 2^E >= the group's largest magnitude) and drops digit pairs below 2^-62 of the scales'
product; the sums carry fp32 rounding only in levels below 2^-56. The bounds below, 2^-46 of
the column-norm product for a Gram entry and 2^-44 of the row-norm times column-norm product
for an update entry (up to 144 terms), hold the FP64 engine too; the double-float engine,
whose splits truncate, gets two bits more.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ENGINES = ["tensor", "df", "f64"]
# bits of the bound below the norm products: the double-float engine keeps about 47 bits per
# product (its splits truncate), two bits fewer than the tensor-core and FP64 engines
GRAM_BITS = {"tensor": 46, "df": 44, "f64": 46}
UPD_BITS = {"tensor": 44, "df": 43, "f64": 44}


@pytest.fixture(scope="module")
def iwf():
    import paper_2404_04507_gb300 as iwf
    assert torch.cuda.is_available()
    return iwf


def _cols(rng, m, n, spread=False):
    X = rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))
    if spread:
        # columns of very different sizes, and entries spanning many decades inside a column
        X *= 10.0 ** rng.uniform(-12, 3, size=(m, 1))
        X *= 10.0 ** rng.uniform(-9, 0, size=(1, n))
    return X


def _dev(X):
    return torch.from_numpy(np.ascontiguousarray(X)).cuda()


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("ma,mb", [(24, 24), (48, 24), (72, 72), (8, 8), (36, 36), (16, 48),
                                   (72, 24), (1, 1), (64, 20), (24, 72)])
@pytest.mark.parametrize("nrows", [1, 17, 4097, 100003])
def test_gram_matches_the_fp64_product(iwf, engine, ma, mb, nrows):
    rng = np.random.default_rng(1000 * ma + mb + nrows)
    A, B = _cols(rng, ma, nrows), _cols(rng, mb, nrows)
    G = iwf.gram(_dev(A), _dev(B), engine=engine).cpu().numpy()
    ref = A.conj() @ B.T
    bound = 2.0 ** -GRAM_BITS[engine] * np.outer(np.linalg.norm(A, axis=1),
                                                 np.linalg.norm(B, axis=1))
    assert np.all(np.abs(G - ref) <= bound), np.max(np.abs(G - ref) / bound)


@pytest.mark.parametrize("engine", ENGINES)
def test_gram_spread_magnitudes_and_zero_columns(iwf, engine):
    rng = np.random.default_rng(7)
    A = _cols(rng, 72, 50000, spread=True)
    B = _cols(rng, 72, 50000, spread=True)
    A[5] = 0.0
    B[70] = 0.0
    A[9, 1234] = 1e6                      # one large entry in an otherwise small column
    G = iwf.gram(_dev(A), _dev(B), engine=engine).cpu().numpy()
    ref = A.conj() @ B.T
    bound = 2.0 ** -GRAM_BITS[engine] * np.outer(np.linalg.norm(A, axis=1),
                                                 np.linalg.norm(B, axis=1))
    assert np.all(np.abs(G - ref) <= bound), np.max(np.abs(G - ref) / np.maximum(bound, 1e-300))
    assert np.all(G[5] == 0) and np.all(G[:, 70] == 0)


def test_gram_hermitian_is_hermitian_to_rounding(iwf):
    rng = np.random.default_rng(3)
    A = _cols(rng, 72, 200000)
    G = iwf.gram(_dev(A), _dev(A)).cpu().numpy()
    n = np.linalg.norm(A, axis=1)
    assert np.all(np.abs(G - G.conj().T) <= 2.0 ** -46 * np.outer(n, n))
    assert np.all(np.abs(np.diag(G).imag) <= 2.0 ** -46 * n * n)


def test_gram_propagates_nan(iwf):
    rng = np.random.default_rng(4)
    A, B = _cols(rng, 24, 5000), _cols(rng, 24, 5000)
    A[3, 17] = np.nan
    G = iwf.gram(_dev(A), _dev(B)).cpu().numpy()
    assert np.all(np.isnan(G[3]))
    assert np.all(np.isfinite(np.delete(G, 3, axis=0)))


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("m,q", [(24, 24), (48, 24), (72, 24), (8, 8), (36, 12), (72, 1),
                                 (5, 3), (72, 16)])
@pytest.mark.parametrize("nrows", [1, 127, 128, 1000, 65537])
def test_update_matches_the_fp64_product(iwf, engine, m, q, nrows):
    rng = np.random.default_rng(100 * m + q + nrows)
    S = _cols(rng, m, nrows)
    C = rng.standard_normal((m, q)) + 1j * rng.standard_normal((m, q))
    Y = iwf.block_update(_dev(S), _dev(C), engine=engine).cpu().numpy()
    ref = (S.T @ C).T
    bound = 2.0 ** -UPD_BITS[engine] * np.outer(np.linalg.norm(C, axis=0),
                                                np.linalg.norm(S, axis=0))
    assert np.all(np.abs(Y - ref) <= bound), np.max(np.abs(Y - ref) / bound)


@pytest.mark.parametrize("engine", ENGINES)
def test_update_subtract_and_spread_rows(iwf, engine):
    rng = np.random.default_rng(11)
    m, q, nrows = 48, 24, 30001
    S = _cols(rng, m, nrows, spread=True)
    C = (rng.standard_normal((m, q)) + 1j * rng.standard_normal((m, q))) * \
        10.0 ** rng.uniform(-6, 2, size=(1, q))
    W0 = _cols(rng, q, nrows)
    Y = _dev(W0.copy())
    iwf.block_update(_dev(S), _dev(C), Y=Y, subtract=True, engine=engine)
    Y = Y.cpu().numpy()
    ref = W0 - (S.T @ C).T
    bound = 2.0 ** -UPD_BITS[engine] * np.outer(np.linalg.norm(C, axis=0),
                                                np.linalg.norm(S, axis=0)) + 2.0 ** -52 * np.abs(W0)
    assert np.all(np.abs(Y - ref) <= bound), np.max(np.abs(Y - ref) / bound)


def test_update_rows_with_zeros_and_nan(iwf):
    rng = np.random.default_rng(12)
    S = _cols(rng, 24, 1000)
    S[:, 10] = 0.0                          # a zero row gives exact zeros
    S[4, 20] = np.nan                       # a NaN row gives NaN outputs in that row only
    C = rng.standard_normal((24, 24)) + 0j
    Y = iwf.block_update(_dev(S), _dev(C)).cpu().numpy()
    assert np.all(Y[:, 10] == 0)
    assert np.all(np.isnan(Y[:, 20]))
    assert np.all(np.isfinite(np.delete(Y, 20, axis=1)))
