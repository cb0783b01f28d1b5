"""The staged check's timeout path, run without any fault: the first bounded
wait of every block is set to give up at once (ne_check_set_wait_limit(0)),
so every block reports NE_ETIMEOUT, reports every position of all of its
units flagged (none was checked), drains its copies (which do arrive) and
returns; the next call with the normal limit checks correctly again."""
import numpy as np
import pytest

import oracle
from paper_1604_04740_gb300 import inputs
from tests.helpers import unpack_flags

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DEV = "cuda"


@pytest.fixture(scope="module")
def ne():
    from paper_1604_04740_gb300 import ne as _ne
    return _ne


@pytest.mark.parametrize("B,M,n", [(64, 3, 1024), (4096, 3, 1024), (300, 4, 2050)])
def test_timed_out_check_reports_every_unit_and_recovers(ne, B, M, n):
    l = 16
    p = ne.params(M, l)
    c = inputs.streams(900 + B, (B, M, n))
    g = inputs.operator_int8(900 + B, (B, n))
    eps = ne.ne_entangle(p, torch.from_numpy(c).to(DEV))
    delta = ne.ne_cconv(p, eps, torch.from_numpy(g).to(DEV), fuse=ne.NE_FUSE_NONE) if n % 64 == 0 else eps
    flags = torch.zeros(ne.flag_words(B, n), dtype=torch.int32, device=DEV)
    nflag = torch.zeros(1, dtype=torch.int64, device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    ne.ne_check_set_wait_limit(0)
    try:
        ne.ne_check(p, delta, 0, flags, nflag, status)
        torch.cuda.synchronize()
    finally:
        ne.ne_check_set_wait_limit()
    assert int(status.item()) == ne.NE_ETIMEOUT
    assert int(nflag.item()) == B * n
    assert unpack_flags(flags.cpu().numpy(), B, n).all()
    # the normal limit: a clean check, and the words still agree with the oracle
    status.zero_()
    ne.ne_check(p, delta, 0, flags, nflag, status)
    assert int(status.item()) == 0 and int(nflag.item()) == 0
    assert not unpack_flags(flags.cpu().numpy(), B, n).any()
    want = oracle.cconv(oracle.entangle(c, l), g) if n % 64 == 0 else oracle.entangle(c, l)
    assert (delta.cpu().numpy() == want).all()


def test_wait_limit_is_validated(ne):
    with pytest.raises(ne.NEError):
        ne.ne_check_set_wait_limit((1 << 22) + 1)
