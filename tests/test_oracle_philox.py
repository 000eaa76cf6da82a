"""Pins for the oracle's Philox4x32-10 and its uniform draw."""
import os

from oracle.philox import draw, philox4x32_10, uniform53

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((tuple(v[0:4]), tuple(v[4:6]), tuple(v[6:10])))
    return rows


def test_known_answer_vectors():
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        assert philox4x32_10(ctr, key) == want


def test_uniform53_range_and_resolution():
    assert uniform53(0, 0) == 0.0
    top = uniform53(0xFFFFFFFF, 0xFFFFFFFF)
    assert top == 1.0 - 2.0 ** -53
    # lowest bit of the 53-bit mantissa comes from bit 6 of w1
    assert uniform53(0, 1 << 6) == 2.0 ** -53
    assert uniform53(0, (1 << 6) - 1) == 0.0
    assert uniform53(1 << 5, 0) == 2.0 ** -27


def test_draw_counter_layout_and_uniformity():
    # distinct (sample, op, purpose) give distinct streams
    a = draw(7, 3, 11, 0)
    b = draw(7, 3, 11, 1)
    c = draw(7, 4, 11, 0)
    d = draw(8, 3, 11, 0)
    assert len({a, b, c, d}) == 4
    # 64-bit sample ids use both counter words
    assert draw(1, 1 << 32, 0, 0) != draw(1, 0, 0, 0)
    # crude uniformity: mean and variance of 20000 draws
    xs = [draw(12345, i, 2, 0) for i in range(20000)]
    m = sum(xs) / len(xs)
    v = sum((x - m) ** 2 for x in xs) / len(xs)
    assert abs(m - 0.5) < 0.01
    assert abs(v - 1.0 / 12.0) < 0.005
