"""Batched form: many systems of uneven sizes in one persistent launch under a
CUDA graph give, per system, exactly the single-system results and the
oracle's."""
import numpy as np
import pytest

import oracle
from paper_1308_4011_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1308_4011_b300 import mmref  # noqa: E402

FIELDS = ("m", "d", "n_improved", "d_lcom_ck_sum", "d_cbo_sum")
SHAPES = [(40, 480, 240), (150, 1800, 900), (1100, 13200, 6600), (7, 30, 10), (2100, 8000, 5000), (300, 3600, 1800)]


def _rows(a):
    return [tuple(int(x[f]) for f in FIELDS) for x in a]


@pytest.fixture(scope="module")
def batch_systems():
    systems = [synth.generate(c, m, a, max_class=80, seed=100 + i) for i, (c, m, a) in enumerate(SHAPES)]
    loaded = [mmref.load_synth(s, device=True, cbo_attrs=(i % 3 != 2)) for i, s in enumerate(systems)]
    yield systems, loaded
    for g in loaded:
        g.free()


def test_batch_equals_single_system_and_oracle(batch_systems):
    systems, loaded = batch_systems
    b = mmref.Batch(loaded, mask=3, min_improved=2, kept_cap=4096)
    dig, nk = b.run()
    dig2, nk2 = b.run()  # graph replay
    assert np.array_equal(dig, dig2) and np.array_equal(nk, nk2)
    for i, (s, g) in enumerate(zip(systems, loaded)):
        d1 = np.zeros(1, dtype=np.uint64)
        mmref.evaluate_moves(g, 3, 2, digest=d1)
        ref = oracle.Oracle(s, cbo_attrs=(i % 3 != 2)).evaluate(mask=3, min_improved=2)
        assert int(dig[i]) == int(d1[0]) == ref.digest, i
        assert nk[i] == ref.n_kept
        top, k = b.suggestions(i, 1000)
        assert k == ref.n_kept
        assert _rows(top) == [tuple(int(x[f]) for f in ("m", "d", "n_improved", "d_ck_sum", "d_cbo_sum"))
                              for x in ref.kept[:1000]]
    b.free()


@pytest.mark.parametrize("tile", [1, 32, 1000, 100000])
def test_batch_tile_sizes_do_not_change_results(batch_systems, tile):
    _, loaded = batch_systems
    b = mmref.Batch(loaded, mask=7, min_improved=1, kept_cap=4096)
    ref = b.run()
    b.set_tile(tile)
    got = b.run()
    assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])
    b.free()


def test_batch_autotune_and_capacity(batch_systems):
    systems, loaded = batch_systems
    b = mmref.Batch(loaded, mask=1, min_improved=1, kept_cap=64)
    chosen = b.autotune()
    assert chosen in (32, 64, 128, 256, 512, 1024)
    tile, blocks = b.config()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert tile == chosen and blocks % sms == 0 and 1 <= blocks // sms <= 8
    dig, nk = b.run()
    for i, s in enumerate(systems):
        ref = oracle.Oracle(s, cbo_attrs=(i % 3 != 2)).evaluate(mask=1, min_improved=1)
        assert nk[i] == ref.n_kept and int(dig[i]) == ref.digest
    big = int(np.argmax(nk))
    assert nk[big] > 64
    with pytest.raises(mmref.MMError) as e:
        b.suggestions(big, 10)
    assert e.value.status == mmref.MM_EBUDGET
    # a system whose kept moves fit still answers
    small = int(np.argmin(nk))
    if nk[small] <= 64:
        top, k = b.suggestions(small, 64)
        ref, kk, _ = mmref.suggest_moves(loaded[small], 64, 1, 1)
        assert k == kk and _rows(top) == _rows(ref)
    b.free()


def test_batch_after_single_calls_recaptures(batch_systems):
    """Other calls on a system may grow its scratch buffers; the batch notices
    and captures its graph again instead of replaying stale pointers."""
    systems, loaded = batch_systems
    b = mmref.Batch(loaded, mask=3, min_improved=2)
    d0, _ = b.run()
    mmref.suggest_moves(loaded[2], 100000, 1, 1)   # large kept list: grows scratch
    rec = torch.empty(loaded[2].n_candidates_full * 16, dtype=torch.uint8, device="cuda")
    mmref.evaluate_moves(loaded[2], 3, 2, records=rec)
    d1, _ = b.run()
    assert np.array_equal(d0, d1)
    b.free()
