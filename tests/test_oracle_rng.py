"""Pins of the checker's random-number layer: Philox4x32-10 against the
published known-answer vectors, exactness of the uniform maps, and the
distributions of the Box-Muller normals and prior draws."""
import numpy as np
import pytest
from scipy import stats

import oracle as O
from conftest import golden_path


def _kat():
    rows = []
    with open(golden_path("philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,want", _kat())
def test_philox_known_answers(ctr, key, want):
    assert O.philox(ctr, key) == want


def test_u24_exact_in_float32_and_open_interval():
    rng = np.random.default_rng(0)
    words = rng.integers(0, 2**32, size=20000, dtype=np.uint64)
    words = np.concatenate([words, [0, 2**32 - 1, 2**31, 511, 512]])
    u = np.array([O.u24(int(w)) for w in words])
    assert np.all(u > 0) and np.all(u < 1)
    assert np.all(u.astype(np.float32).astype(np.float64) == u)
    # odd multiples of 2^-24
    k = u * 2**24
    assert np.all(k == np.round(k)) and np.all(k.astype(np.int64) % 2 == 1)


def test_u53_exact_and_open_interval():
    assert O.u53(0, 0) == 2.0**-53
    assert O.u53(2**32 - 1, 2**32 - 1) == 1.0 - 2.0**-53
    k = O.u53(12345678, 87654321) * 2.0**53
    assert k == np.round(k) and int(k) % 2 == 1


def test_philox_words_uniform():
    words = [w for c in range(4000) for w in O.philox([c, 7, 3, 0], [11, 13])]
    u = np.array([O.u24(w) for w in words])
    assert stats.kstest(u, "uniform").pvalue > 1e-3


def test_box_prior_draws_uniform_and_gauss_prior_draws_normal():
    d = 3
    box = O.Problem(("box", np.zeros(d), np.full(d, 2.0)), "flat")
    xs = np.array([_draw(box, s) for s in range(3000)])
    for i in range(d):
        assert stats.kstest(xs[:, i] / 2.0, "uniform").pvalue > 1e-3
    g = O.Problem(("gauss", np.full(d, 1.0), np.full(d, 3.0)), "flat")
    xs = np.array([_draw(g, s) for s in range(3000)])
    for i in range(d):
        assert stats.kstest((xs[:, i] - 1.0) / 3.0, "norm").pvalue > 1e-3
    # independent coordinates from the same Box-Muller pair
    r = np.corrcoef(xs[:, 0], xs[:, 1])[0, 1]
    assert abs(r) < 4.0 / np.sqrt(3000)


def _draw(pb, slot):
    import ctypes as C
    x = np.empty(pb.d)
    O.lib().orc_prior_draw(C.byref(pb.s), 5, 0, slot, O._d(x))
    return x


def test_counter_and_key_layout_of_the_initial_draw():
    """Reading C14: key = (seed_lo, seed_hi XOR run_id), counter (0, slot,
    TAG_INIT, word / 4) for the prior draw.  The box draw a + (b - a) u24(w)
    is rebuilt here from the known-answer-pinned generator, word by word, so a
    wrong key (a dropped run id), counter or word index fails."""
    d, m = 5, 6
    seed, run_id = (7 << 32) | 123456789, 37
    a, b = np.linspace(-1.0, 0.0, d), np.linspace(1.0, 3.0, d)
    pb = O.Problem(("box", a, b), "flat")
    x, _, _ = O.init_live(pb, O.make_opts(m, 1, 1, seed=seed, run_id=run_id))
    key = [seed & 0xFFFFFFFF, (seed >> 32) ^ run_id]
    tag_init = 0xFFFFFFF1
    for slot in range(m):
        for i in range(d):
            w = O.philox([0, slot, tag_init, i // 4], key)[i % 4]
            assert x[slot, i] == a[i] + (b[i] - a[i]) * O.u24(w)
    # a different run id gives a different stream
    x2, _, _ = O.init_live(pb, O.make_opts(m, 1, 1, seed=seed, run_id=run_id + 1))
    assert not np.array_equal(x, x2)
