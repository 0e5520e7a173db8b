"""FP64 products on the tensor cores (exact integer slices): C = A B^T through
ltmp2_dgemm_nt against the product in long double, on ragged shapes (not multiples of the
128 x 64 x 16 tiles), a zero row, rows of very different magnitude and mixed signs.  The
bound is the scheme's: K x 2^-52 x max_k |a_ik| x max_k |b_jk| per element, the size of an
FP64 dot product's own rounding bound for rows of even magnitude."""
import numpy as np
import pytest

import paper_1611_06797_gb300 as L

pytestmark = pytest.mark.gpu


def _case(m, n, k, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((m, k))
    b = rng.standard_normal((n, k))
    a *= 10.0 ** rng.uniform(-60, 60, size=(m, 1))       # rows of very different magnitude
    b *= 10.0 ** rng.uniform(-60, 60, size=(n, 1))
    a[3] = 0.0                                            # a zero row
    a[5, ::7] *= 1e-12                                    # small entries inside a row
    return a, b


@pytest.mark.parametrize("m,n,k,seed", [(300, 200, 1000, 1), (128, 64, 16, 2), (129, 65, 17, 3),
                                        (256, 130, 3071, 4)])
def test_dgemm_matches_long_double(m, n, k, seed):
    import torch
    a, b = _case(m, n, k, seed)
    c = L.ltmp2_dgemm_nt(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()).cpu().numpy()
    ref = a.astype(np.longdouble) @ b.astype(np.longdouble).T
    bound = k * 2.0 ** -52 * np.abs(a).max(axis=1)[:, None] * np.abs(b).max(axis=1)[None, :]
    err = np.abs(c.astype(np.longdouble) - ref)
    assert np.all(err <= bound), float((err / np.maximum(bound, 1e-300)).max())
    assert np.all(c[3] == 0.0)
    # as accurate as the FP64 product itself, element by element, within a factor
    c64 = a @ b.T
    err64 = np.abs(c64.astype(np.longdouble) - ref)
    assert float(err.max()) <= 16.0 * float(err64.max())


def test_dgemm_arguments():
    import torch
    a = torch.zeros((4, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        L.ltmp2_dgemm_nt(a.float(), a)
    with pytest.raises(ValueError):
        L.ltmp2_dgemm_nt(a, torch.zeros((4, 9), dtype=torch.float64, device="cuda"))
    c = L.ltmp2_dgemm_nt(a, a)
    assert c.shape == (4, 4) and float(c.abs().max()) == 0.0
