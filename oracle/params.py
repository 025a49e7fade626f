"""NTT-friendly primes and roots of unity (oracle; test infrastructure only).

Sec. II-A asks for a prime q with a primitive N-th (here 2N-th, for the
negacyclic form of Eq. (4)) root of unity psi, obtained from a generator as
g^((q-1)/N). The paper fixes no particular primes or generator, so this module
fixes one deterministic reading:

* primes: q = 1 (mod 2^(logn_max+1)), 2^29 < q < 2^30, enumerated in
  descending order starting just below 2^30;
* psi: x = the smallest integer >= 2 that is a quadratic non-residue mod q,
  psi_N = x^((q-1)/(2N)) mod q. Then psi^N = x^((q-1)/2) = -1, so psi has order
  exactly 2N, and psi_(N/2) = psi_N^2 for every N.

Primality is decided by the deterministic Miller-Rabin test with bases
2, 3, 5, 7, which is exact for every n < 3,215,031,751 (> 2^31).
"""


def is_prime(n: int) -> bool:
    """Deterministic Miller-Rabin, exact for n < 3,215,031,751."""
    if n < 2:
        return False
    for p in (2, 3, 5, 7, 11, 13):
        if n % p == 0:
            return n == p
    if n >= 3_215_031_751:
        raise ValueError("is_prime: bases 2,3,5,7 are exact only below 3,215,031,751")
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in (2, 3, 5, 7):
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def ntt_primes(count: int, logn_max: int = 16, bits: int = 30) -> list:
    """The first `count` primes q = 1 mod 2^(logn_max+1) below 2^bits, descending."""
    step = 1 << (logn_max + 1)
    q = ((1 << bits) - 1) // step * step + 1
    out = []
    while len(out) < count:
        if q <= (1 << (bits - 1)):
            raise ValueError("ran out of primes in (2^(bits-1), 2^bits)")
        if is_prime(q):
            out.append(q)
        q -= step
    return out


def default_moduli(n_q: int = 44, n_p: int = 8, logn_max: int = 16):
    """Special primes p_0..p_{n_p-1} are the n_p largest; q_0.. the next n_q.

    Returns (q_list, p_list), both descending.
    """
    allp = ntt_primes(n_q + n_p, logn_max)
    return allp[n_p:], allp[:n_p]


def nonresidue(q: int) -> int:
    x = 2
    while pow(x, (q - 1) // 2, q) != q - 1:
        x += 1
    return x


def psi(q: int, n: int) -> int:
    """Primitive 2N-th root of unity mod q (N = n)."""
    if (q - 1) % (2 * n):
        raise ValueError("q != 1 mod 2N")
    return pow(nonresidue(q), (q - 1) // (2 * n), q)
