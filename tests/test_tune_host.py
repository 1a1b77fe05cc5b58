"""Host-side logic of the kernel autotuner's table: loading, validation and
saving of the JSON-lines file (no GPU needed: these calls never touch a
device)."""
import json

import pytest


@pytest.fixture()
def btas():
    import paper_1701_04733_gb300 as b
    b.build()
    b.lib()
    b.tune_clear()
    yield b
    b.tune_clear()


def _line(**kv):
    e = {"arch": 103, "sms": 152, "semiring": 0, "dtype": 0, "m_bucket": 13, "n_bucket": 13, "k_bucket": 13,
         "variant": 1, "ns": 4, "cfg": 4, "group_m": 8, "candidates": 17, "tile_m": 128, "tile_n": 128,
         "seconds": 0.0302, "terms_per_second": 1.82e13}
    e.update(kv)
    return json.dumps(e)


def test_load_save_roundtrip(btas, tmp_path):
    lines = [_line(),
             _line(semiring=1, dtype=1, variant=2, ns=0, cfg=4, group_m=4, seconds=0.0297),
             _line(dtype=2, variant=16, ns=5, cfg=0, tile_n=256, m_bucket=12, n_bucket=12, k_bucket=12),
             _line(arch=100, sms=148, m_bucket=10)]  # another device's entry is kept
    src = tmp_path / "in.jsonl"
    src.write_text("\n".join(lines) + "\n\n")
    assert btas.tune_load(str(src)) == 4
    assert btas.tune_entries() == 4
    out = tmp_path / "out.jsonl"
    btas.tune_save(str(out))
    got = sorted((json.loads(x) for x in out.read_text().splitlines()), key=json.dumps)
    want = sorted((json.loads(x) for x in lines), key=json.dumps)
    assert len(got) == len(want)
    for g, w in zip(sorted(got, key=lambda d: tuple(d[k] for k in sorted(d) if k != "seconds")),
                    sorted(want, key=lambda d: tuple(d[k] for k in sorted(d) if k != "seconds"))):
        assert set(g) == set(w)
        for k in w:
            assert g[k] == pytest.approx(w[k], rel=1e-8), k
    # the same key loaded again replaces, not duplicates
    assert btas.tune_load(str(src)) == 4
    assert btas.tune_entries() == 4
    btas.tune_clear()
    assert btas.tune_entries() == 0


@pytest.mark.parametrize("bad,why", [
    ("not json at all", "is not a tuning entry"),
    (_line(cfg=99), "does not have"),                 # no such tile configuration
    (_line(variant=2, ns=0), "does not have"),        # fp32 kernel under an int32 key
    (_line(dtype=2, variant=16, ns=3), "does not have"),  # u16 split that is not compiled
    (_line(dtype=2, semiring=1, variant=16, ns=5), "does not have"),  # u16 is min-plus only
    (_line(group_m=0), "does not have"),
])
def test_malformed_file_adds_nothing(btas, tmp_path, bad, why):
    p = tmp_path / "bad.jsonl"
    p.write_text(_line() + "\n" + bad + "\n")
    with pytest.raises(btas.BtasError) as ei:
        btas.tune_load(str(p))
    assert ei.value.status == 1
    assert "line 2" in str(ei.value) and why in str(ei.value)
    assert btas.tune_entries() == 0


def test_missing_file_and_empty_path(btas, tmp_path):
    with pytest.raises(btas.BtasError):
        btas.tune_load(str(tmp_path / "nope.jsonl"))
    assert btas.btas_tune_save("") == 1
    assert btas.btas_tune_load("", None) == 1


def test_tune_gemm_argument_errors(btas):
    """Rejected on the host before any device call."""
    assert btas.btas_tune_gemm(5, 0, 8, 8, 8, None, None) == 1   # semiring
    assert btas.btas_tune_gemm(0, 9, 8, 8, 8, None, None) == 1   # dtype
    assert btas.btas_tune_gemm(0, 0, 0, 8, 8, None, None) == 1   # empty
    assert btas.btas_tune_gemm(1, 2, 8, 8, 8, None, None) == 7   # u16 max-plus
