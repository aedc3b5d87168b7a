"""Eq. 1 takes the hash modulo V.  Tables whose V is not a power of two take
that modulo by an exact division by an invariant integer on the device (one
32-bit high multiply).  The oracle takes a plain %.  These builds compare the
two, byte for byte, at divisors where a wrong shift or constant would show:
small odd and even ones, one above and one below a power of two, and large
ones up to 2^27 + 1."""
import numpy as np
import pytest

from paper_1907_02900_gb300 import datagen as dg
from gpu_util import table_np, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("V", [3, 6, 641, (1 << 20) + 1, (1 << 24) - 1, 3 * (1 << 25) + 1, (1 << 27) + 1])
@pytest.mark.parametrize("kt", ["u32", "u64"])
def test_build_at_divisor_edges(hg, orc, V, kt):
    n = 1 << 18
    keys = dg.uniform_keys_u32(n, 61) if kt == "u32" else dg.uniform_keys_u64(n, 61)
    t = hg.build(to_dev(keys), V, seed=5)
    off, ck, ci = table_np(t)
    roff, rk, ri = orc.build(keys, V, 5)
    assert np.array_equal(off, roff) and np.array_equal(ck, rk) and np.array_equal(ci, ri)
    q = dg.queries_u32(n, keys, 0.5, 62) if kt == "u32" else dg.queries_u64(n, keys, 0.5, 62)
    for binned in (False, True):
        assert np.array_equal(to_np(hg.probe(t, to_dev(q), binned=binned)), orc.probe(roff, rk, q, V, 5))
