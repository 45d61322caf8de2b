"""The paper's own test family (Sec. 3, Table 1): m = 2n, r = 7n/8, entries
from U[-1,1] factors, n = 32 .. 1024.  The GPU's G+ must have the oracle's
rank, match the oracle within the bar of its mode, and meet the paper's
accuracy statement: every coefficient of the four Penrose error matrices at
most 2e-10 in absolute value.  Where the oracle itself does not meet 2e-10 on
our instance of the family (n = 1024, seed 1024: kept block close to
singular, residual 4.7e-9 with the correctly rounded Gram matrix, 3.7e-8
with an FP64 one), the GPU is held to 4x the oracle's residual or 8x that of
the oracle with an FP64 Gram matrix, whichever is larger."""
import numpy as np
import pytest

import oracle
from paper_0804_4809_gb300 import inputs
from tests.gpu_util import rel, tol_for, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", ["fp64", "exact"])
@pytest.mark.parametrize("n", [32, 64, 128, 256, 512, 1024])
def test_paper_family(n, mode):
    from paper_0804_4809_gb300 import cpinv
    G = inputs.paper_family(n, seed=n)
    Y, r = cpinv.pinv(to_dev(G), mode=mode)
    Y = Y.cpu().numpy()
    Yo, fac = oracle.geninv(G, return_factors=True)
    assert r == fac["rank"] == 7 * n // 8
    # the stated bar, or 8x the oracle's own change between a correctly
    # rounded and an FP64 Gram matrix where the kept block is close to
    # singular (n = 1024: smallest kept pivot 2.6e3 tol, change 9.4e-10)
    Yf = oracle.geninv(G, exact_gram=False)
    sens = rel(Yf, Yo)
    assert rel(Y, Yo) <= max(tol_for(mode, G, r), 8.0 * sens), (rel(Y, Yo), sens)
    res = oracle.penrose_residuals(G, Y)
    res_o = oracle.penrose_residuals(G, Yo)
    res_f = oracle.penrose_residuals(G, Yf)
    for k, v in res.items():
        if k.endswith(":max"):
            assert v <= max(2e-10, 4.0 * res_o[k], 8.0 * res_f[k]), (k, v, res_o[k], res_f[k])
