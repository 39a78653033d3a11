"""Pins of the oracle's Sobol' generator and randomisation (CPU only).

Every check here is a property fixed by the mathematics of Sec. 2.2 (van der
Corput radical inverse, primitive polynomials, digital nets), not a retyping of
the oracle's own formulas.
"""
import itertools

import numpy as np
import pytest

SEED = 0x220911337


def euler_phi(n: int) -> int:
    result, p, m = n, 2, n
    while p * p <= m:
        if m % p == 0:
            while m % p == 0:
                m //= p
            result -= result // p
        p += 1
    if m > 1:
        result -= result // m
    return result


def test_primitive_polynomials_textbook_list(oracle_lib):
    # Sec. 2.2.2: the primitive polynomials of degree <= 5 over GF(2), as
    # integers (bit i = coefficient of x^i): x+1, x^2+x+1, x^3+x+1, x^3+x^2+1,
    # x^4+x+1, x^4+x^3+1 and the six quintics.
    expected = [3, 7, 11, 13, 19, 25, 37, 41, 47, 55, 59, 61]
    assert list(oracle_lib.primitive_polys(12)) == expected


def test_primitive_polynomial_count_per_degree(oracle_lib):
    # There are phi(2^q - 1)/q primitive polynomials of degree q.
    want = {q: euler_phi(2 ** q - 1) // q for q in range(1, 11)}
    polys = oracle_lib.primitive_polys(sum(want.values()))
    degs = [int(p).bit_length() - 1 for p in polys]
    for q, c in want.items():
        assert degs.count(q) == c, q
    assert degs == sorted(degs)


def test_direction_integers_odd_and_bounded(oracle_lib):
    # m_i odd and < 2^i for every i (Sec. 2.2.2), for all dims up to d=365.
    v = oracle_lib.direction_numbers(364).astype(np.uint64)
    for i in range(1, 33):
        m = v[:, i - 1] >> np.uint64(32 - i)
        assert np.all(m & np.uint64(1) == 1)
        assert np.all(m < (np.uint64(1) << np.uint64(i)))
        assert np.all(v[:, i - 1] == (m << np.uint64(32 - i)))


def radical_inverse_bits(k: int) -> int:
    # psi_2(k) (eq. RadicalInverseFunction) as a 32-bit binary fraction.
    y = 0
    for j in range(32):
        if (k >> j) & 1:
            y |= 1 << (31 - j)
    return y


def test_dimension_one_is_van_der_corput(oracle_lib):
    ks = list(range(4096)) + [2 ** 20 + 12345, 2 ** 31 + 7, 2 ** 32 - 1]
    for k in ks[::97] + ks[-3:]:
        y = oracle_lib.sobol(SEED, 0, 1, k, 1, scrambled=False, gray=False)[0, 0]
        assert int(y) == radical_inverse_bits(k)
    y = oracle_lib.sobol(SEED, 0, 1, 0, 4096, scrambled=False, gray=False)[:, 0]
    assert [int(a) for a in y] == [radical_inverse_bits(k) for k in range(4096)]


def t_value(bits: np.ndarray, m: int) -> int:
    """Smallest t such that the 2^m points form a (t, m, s)-net in base 2."""
    s = bits.shape[1]
    for t in range(m + 1):
        good = True
        for comp in itertools.product(range(m - t + 1), repeat=s):
            if sum(comp) != m - t:
                continue
            keys = np.zeros(len(bits), dtype=np.int64)
            for j, c in enumerate(comp):
                if c:
                    keys = keys * (1 << c) + (bits[:, j] >> np.uint32(32 - c)).astype(np.int64)
            if not np.all(np.bincount(keys, minlength=1 << (m - t)) == (1 << t)):
                good = False
                break
        if good:
            return t
    return m


@pytest.mark.parametrize("scrambled", [False, True])
def test_net_quality_first_dimensions(oracle_lib, scrambled):
    # Sobol's bound t <= sum_j (deg p_j - 1): dims 1,2 form a (0,m,2)-net,
    # dims 1..3 a (1,m,3)-net, dims 1..5 a (5,m,5)-net.  A linear scramble
    # with unit diagonal plus a digital shift keeps the t-value.
    bound = {2: 0, 3: 1, 4: 3, 5: 5}
    for s, m in [(2, 6), (2, 10), (3, 8), (4, 8), (5, 8)]:
        bits = oracle_lib.sobol(SEED, 3, s, 0, 1 << m, scrambled=scrambled, gray=True)
        assert t_value(bits, m) <= bound[s], (s, m)


@pytest.mark.parametrize("scrambled", [False, True])
def test_dyadic_blocks_stratify_every_coordinate(oracle_lib, scrambled):
    # Each block {k : floor(k / 2^m) = c} has one point in each interval
    # [i/2^m, (i+1)/2^m) of every coordinate (a nonsingular upper-triangular
    # generator per dimension; preserved by L C and the shift).
    n = 63
    for m, c in [(4, 0), (7, 0), (7, 5), (10, 3)]:
        bits = oracle_lib.sobol(SEED, 1, n, c << m, 1 << m, scrambled=scrambled, gray=False)
        top = bits >> np.uint32(32 - m)
        for j in range(n):
            assert np.array_equal(np.sort(top[:, j]), np.arange(1 << m)), (m, c, j)


def test_gray_order_gives_the_same_point_set(oracle_lib):
    for m in (5, 9):
        a = oracle_lib.sobol(SEED, 2, 15, 0, 1 << m, scrambled=True, gray=True)
        b = oracle_lib.sobol(SEED, 2, 15, 0, 1 << m, scrambled=True, gray=False)
        ka = sorted(map(tuple, a.tolist()))
        kb = sorted(map(tuple, b.tolist()))
        assert ka == kb


def test_gray_consecutive_points_differ_by_one_direction_number(oracle_lib):
    # g(k+1) = g(k) ^ 2^c with c = ctz(k+1), so y(k+1) ^ y(k) = L v_{c+1}
    # (the shift cancels): the XOR of consecutive scrambled points equals the
    # XOR of points g=0 and g=2^c.
    n = 7
    pts = oracle_lib.sobol(SEED, 4, n, 0, 1024, scrambled=True, gray=True)
    nat = oracle_lib.sobol(SEED, 4, n, 0, 1024, scrambled=True, gray=False)
    for k in range(1023):
        c = ((k + 1) & -(k + 1)).bit_length() - 1
        assert np.array_equal(pts[k + 1] ^ pts[k], nat[1 << c] ^ nat[0])


def test_scramble_is_affine_with_unit_lower_triangular_matrix(oracle_lib):
    for r, j in [(0, 0), (3, 17), (31, 363)]:
        rows, shift = oracle_lib.scramble(SEED, r, j)
        for i in range(1, 33):
            diag = 1 << (32 - i)
            assert int(rows[i - 1]) & diag
            assert int(rows[i - 1]) & (diag - 1) == 0  # nothing below the diagonal digit
    # point with index 0 is y = 0, so its scrambled value is the shift itself
    for r in (0, 9):
        first = oracle_lib.sobol(SEED, r, 40, 0, 1, scrambled=True, gray=True)[0]
        shifts = [oracle_lib.scramble(SEED, r, j)[1] for j in range(40)]
        assert [int(x) for x in first] == shifts
    # affine: s(y1 ^ y2) = s(y1) ^ s(y2) ^ e
    nat_u = oracle_lib.sobol(SEED, 6, 5, 0, 64, scrambled=False, gray=False)
    nat_s = oracle_lib.sobol(SEED, 6, 5, 0, 64, scrambled=True, gray=False)
    e = nat_s[0]
    for a, b in [(3, 5), (17, 40), (63, 1)]:
        assert np.array_equal(nat_u[a] ^ nat_u[b], nat_u[a ^ b])
        assert np.array_equal(nat_s[a] ^ nat_s[b] ^ e, nat_s[a ^ b])


def test_scramble_bits_look_uniform(oracle_lib):
    # Each random bit of L and e is a fair coin: over 64 replicates x 64 dims
    # every bit position is set close to half the time.
    shifts = np.array([oracle_lib.scramble(SEED, r, j)[1] for r in range(64) for j in range(64)],
                      dtype=np.uint64)
    for b in range(32):
        frac = np.mean((shifts >> np.uint64(b)) & np.uint64(1))
        assert 0.45 < frac < 0.55, b
    # replicates differ
    a = oracle_lib.sobol(SEED, 0, 8, 0, 16)
    b = oracle_lib.sobol(SEED, 1, 8, 0, 16)
    c = oracle_lib.sobol(SEED + 1, 0, 8, 0, 16)
    assert not np.array_equal(a, b) and not np.array_equal(a, c)
