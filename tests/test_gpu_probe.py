"""The issue-rate probe (btas_measure_issue_rate_ex): every instruction mix
runs at 1 and 2 CTAs per SM and reports a rate inside the physical range of
the SM (at most 4 schedulers x 32 lanes x 2 terms per instruction for the
packed mix, 128 x 1 or x 2 for the others).  The rates themselves are
measurements, not checked here."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def btas():
    import torch
    import paper_1701_04733_gb300 as b
    assert torch.cuda.is_available()
    b.lib()
    return b


@pytest.mark.parametrize("ctas", [1, 2])
def test_every_mix_reports_a_physical_rate(btas, ctas):
    for mix in range(16):
        r = btas.measure_issue_rate(mix, ctas)
        limit = 256.0 if mix == 2 else 128.0 * 2
        assert 1.0 < r <= limit, (mix, ctas, r)
