"""The per-kernel profiler's algorithmic flops (the numerator of the
benchmark's roofline): summed over one call they equal the executed count of
the algorithm up to the panel factorizations' lower-order work, which the
panel kernels do not count."""
import pytest
import torch

from paper_2208_01239_gb300 import flops
from paper_2208_01239_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_2208_01239_gb300 import build, frob
    build.build()
    frob.load()
    return frob


@pytest.mark.parametrize("op,alg,n", [("frob_inv", "frob_lu", 1088), ("cplx_lu_inv", "cplx_lu", 1088),
                                      ("frob_inv", "frob_lu", 320)])
def test_profile_flops_match_executed_count(F, op, alg, n):
    dm = torch.from_numpy(W.gaussian(n, 1, seed=11)).cuda()
    f = getattr(F, op)
    f(dm)
    torch.cuda.synchronize()
    F.profile_enable(True)
    f(dm)
    torch.cuda.synchronize()
    F.profile_enable(False)
    rep = F.profile_report()
    counted = sum(v[2] for v in rep.values())
    want = flops.executed(alg, n)
    # uncounted: the panels and the U12 solves beside them (about 2 x 32 n^2
    # flops each per factorization) and the triangular inverses' 64 x 64
    # diagonal blocks; counted beyond the leading order: whole 64 x 64 tiles
    # on the diagonals of the triangular products, and, in FP64 from order
    # 256 on, the zero triangles of the triangular inverse's joins, which run
    # as full products on the tensor cores (at most n^3 / 3 more), and, above
    # order 512, the recursive LU's U12 = (L11^{-1}) A12 in place of a solve
    # (per block split, 2 w1^3 / 3 for the inverse and w1^2 (w - w1) more for
    # the product: at most about n^3 / 6 over both factorizations), and, from
    # order 1024 on, the recursive triangular solves' diagonal blocks of up to
    # 256 rows as full products with the blocks' inverses (256^2 nrhs more per
    # block of 256 rows, 256 n^2 per solve, three solves)
    hi = 1.03
    if alg == "frob_lu" and n >= 256:
        hi += (1 / 3) / float(flops.EXECUTED[alg])
    if alg == "frob_lu" and n > 512:
        hi += (1 / 6) / float(flops.EXECUTED[alg])
    if alg == "frob_lu" and n >= 1024:
        hi += 3 * 256 / n / float(flops.EXECUTED[alg])
    assert 0.90 * want <= counted <= hi * want, (counted / want, rep)
    assert all(v[1] > 0 for v in rep.values())
