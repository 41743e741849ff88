/*
 * Philox4x64-10 counter-based generator, written from its published definition
 * (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 * SC'11, Section 4: the Philox S-box with 2 multipliers, Weyl key schedule and
 * 10 rounds).  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Pinned against numpy.random.Philox (an independent implementation of the same
 * definition) in tests/test_oracle_rng.py.
 */
#include "oracle.h"

/* Round multipliers and key increments of Philox4x64 (Salmon et al. 2011). */
static const uint64_t PHILOX_M0 = 0xD2E7470EE14C6C93ull;
static const uint64_t PHILOX_M1 = 0xCA5A826395121157ull;
static const uint64_t PHILOX_W0 = 0x9E3779B97F4A7C15ull;
static const uint64_t PHILOX_W1 = 0xBB67AE8584CAA73Bull;

static void mulhilo(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 r = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(r >> 64);
    *lo = (uint64_t)r;
}

void or_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo(PHILOX_M0, x0, &hi0, &lo0);
        mulhilo(PHILOX_M1, x2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ x1 ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ x3 ^ k1;
        uint64_t n3 = lo0;
        x0 = n0; x1 = n1; x2 = n2; x3 = n3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}
