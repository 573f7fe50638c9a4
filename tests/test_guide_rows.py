"""Guide tables of the FP32 jump samplers (host code of the C ABI, no GPU).

The FP32 form inverts the jump distributions of Eq. update_evib through
per-cell cumulative rows and, per row, a guide of 256 bytes (Chen & Asau's
indexed search): one byte per bin of a 23-bit uniform's top eight bits.  A
byte answers the lookup outright (bit 7: the outcome) when no row entry lies
inside its bin, else gives the count to start from.  Two checks:
  * against the definition written out per bin (float64 bin bounds, prefix
    counts), byte for byte;
  * against what a lookup means: for every uniform u = (2 i + 1) 2^-24 of
    sampled indices i, the byte's answer equals the number of row entries
    <= u (n - that number for a flipped binomial row).
Rows: pmf recursions of the NB and binomial jumps in float32 and adversarial
rows with entries on and next to bin bounds, clusters inside one bin,
entries below the smallest uniform, +inf tails and an underflowed P(0).
"""
import numpy as np
import pytest

from paper_2508_05642_gb300 import usp

KJK, KGB = 48, 256


def _bounds(m):
    umin = (2.0 * (m << 15) + 1.0) * 2.0 ** -24
    umax = (2.0 * ((m << 15) + 32767) + 1.0) * 2.0 ** -24
    return umin, umax


def _guide_by_definition(row, n_flip):
    row = np.asarray(row, dtype=np.float32).astype(np.float64)
    if row[0] < 0:
        return np.full(KGB, 0xFF, dtype=np.uint8)
    g = np.zeros(KGB, dtype=np.uint8)
    for m in range(KGB):
        umin, umax = _bounds(m)
        k = 0
        while k < KJK and row[k] <= umin:
            k += 1
        exact = k >= KJK or row[k] > umax
        o = n_flip - k if (exact and k < KJK and n_flip >= 0) else k
        g[m] = o | (0x80 if exact else 0)
    return g


def _count(row, u):
    """Number of leading row entries <= u (the sequential search's k)."""
    k = 0
    while k < KJK and row[k] <= u:
        k += 1
    return k


def _nb_row(r, p):
    q = np.float32(1.0) - np.float32(p)
    P = np.float32(p) ** np.int32(r)
    T = np.full(KJK, np.inf, dtype=np.float32)
    cdf = P
    T[0] = cdf
    for j in range(1, KJK):
        k = j - 1
        P = np.float32(P * np.float32(np.float32(k + r) / np.float32(k + 1)))
        P = np.float32(P * q)
        nc = np.float32(cdf + P)
        if nc == cdf:
            break
        cdf = nc
        T[j] = cdf
    return T


def _b_row(n, p):
    q = np.float32(1.0) - np.float32(p)
    P = q ** np.int32(n)
    pq = np.float32(np.float32(p) / q)
    T = np.full(KJK, np.inf, dtype=np.float32)
    cdf = P
    T[0] = cdf
    for j in range(1, min(n, KJK)):
        k = j - 1
        P = np.float32(P * np.float32(np.float32(n - k) / np.float32(k + 1)))
        P = np.float32(P * pq)
        nc = np.float32(cdf + P)
        if nc == cdf:
            break
        cdf = nc
        T[j] = cdf
    return T


def _adversarial_rows(rng):
    rows = []
    # entries exactly on bin bounds and one float step either side
    for m in (0, 1, 7, 100, 128, 254, 255):
        umin, umax = _bounds(m)
        for v in (umin, umax):
            for d in (-1, 0, 1):
                e = np.nextafter(np.float32(v), np.float32(np.inf if d > 0 else -np.inf)) if d else np.float32(v)
                T = np.full(KJK, np.inf, dtype=np.float32)
                T[0] = np.float32(min(e, 0.5 * umin)) if m > 0 else np.float32(1e-9)
                T[1] = e
                T[2] = np.float32(min(1.0 - 2.0 ** -24, umax + 0.01))
                T[:3] = np.sort(T[:3])
                rows.append(T)
    # clusters of several entries inside one bin, then a gap
    for m in (3, 200, 255):
        umin, umax = _bounds(m)
        T = np.full(KJK, np.inf, dtype=np.float32)
        vals = np.sort(rng.uniform(umin, umax, 5)).astype(np.float32)
        T[:5] = vals
        rows.append(T)
    # entries below the smallest uniform 2^-24
    T = np.full(KJK, np.inf, dtype=np.float32)
    T[:4] = np.array([1e-12, 3e-9, 5e-8, 0.3], dtype=np.float32)
    rows.append(T)
    # 48 finite entries (the search runs past the row near u = 1)
    T = np.sort(rng.uniform(0.0, 0.999, KJK)).astype(np.float32)
    rows.append(T)
    # random monotone rows with +inf tails
    for _ in range(30):
        n = int(rng.integers(1, KJK + 1))
        T = np.full(KJK, np.inf, dtype=np.float32)
        T[:n] = np.sort(rng.uniform(0.0, 1.0, n) ** rng.uniform(0.2, 5.0)).astype(np.float32)
        rows.append(T)
    # underflowed P(0)
    T = np.full(KJK, np.inf, dtype=np.float32)
    T[0] = -1.0
    rows.append(T)
    return rows


def _all_rows():
    rng = np.random.default_rng(11)
    rows = [(_nb_row(r, p), -1) for r in (1, 2, 5, 12, 32) for p in (0.05, 0.4, 0.8, 0.97, 0.999)]
    rows += [(_b_row(n, p), -1) for n in (1, 2, 6, 17, 31) for p in (0.01, 0.2, 0.45)]
    rows += [(_b_row(n, 1.0 - p), n) for n in (1, 3, 9, 31) for p in (0.55, 0.8, 0.99)]
    rows += [(T, -1) for T in _adversarial_rows(rng)]
    # flipped binomial rows end at n: the entries from n on are +inf
    for T in _adversarial_rows(np.random.default_rng(12))[:12]:
        n = int(rng.integers(1, 32))
        T = T.copy()
        T[n:] = np.inf
        rows.append((T, n))
    return rows


def test_guide_bytes_match_their_definition():
    for row, nf in _all_rows():
        assert np.array_equal(usp.usp_guide_row(row, nf), _guide_by_definition(row, nf)), (row[:6], nf)


def test_guide_lookups_equal_the_row_search():
    rng = np.random.default_rng(3)
    for row, nf in _all_rows():
        g = usp.usp_guide_row(row, nf)
        if row[0] < 0:
            assert np.all(g == 0xFF)
            continue
        # every bin's two ends and random indices inside
        idx = np.concatenate([np.arange(KGB) << 15, (np.arange(KGB) << 15) + 32767,
                              rng.integers(0, 1 << 23, 4000)])
        for i in idx:
            u = np.float32((2.0 * int(i) + 1.0) * 2.0 ** -24)
            k = _count(row, u)
            b = int(g[int(i) >> 15])
            if b & 0x80:
                o = b & 0x7F
                if o >= KJK:
                    assert k >= KJK or b == 0xFF      # the sequential search decides
                else:
                    assert o == (nf - k if nf >= 0 else k)
            else:
                # the search from kk: the entries before it are all <= u
                kk = b & 0x7F
                assert kk <= k and all(row[j] <= u for j in range(kk))


def test_guide_row_rejects_bad_arguments():
    row = np.full(KJK, np.inf, dtype=np.float32)
    row[0] = 0.5
    with pytest.raises(RuntimeError):
        usp.usp_guide_row(row, 32)
    with pytest.raises(RuntimeError):
        usp.usp_guide_row(row, -2)
    with pytest.raises(ValueError):
        usp.usp_guide_row(row[:10])
    # a flipped binomial row n must end at n (row[n] = +inf)
    row2 = row.copy()
    row2[:4] = [0.1, 0.2, 0.3, 0.4]
    with pytest.raises(RuntimeError):
        usp.usp_guide_row(row2, 2)
    usp.usp_guide_row(row2, 4)
