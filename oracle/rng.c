/*
 * Oracle: Philox4x32-10 — TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Written from the published definition of Philox4x32 with 10 rounds (Salmon et al., "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11): each round multiplies counter words 0 and 2 by the two round
 * multipliers, XORs the high halves with the other two counter words and the round key, and permutes;
 * the key is advanced by the two Weyl increments between rounds.
 *
 * The method draws its random numbers (free paths Sec. 3.1, roulette Sec. 3.1, HG sampling Eq. 1,
 * latent and posterior normals Sec. 3.2) from this stream; the CUDA library implements the same published
 * generator independently.
 */
#include "oracle.h"

void om_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod_a = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t prod_b = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi_a = (uint32_t)(prod_a >> 32), lo_a = (uint32_t)prod_a;
        uint32_t hi_b = (uint32_t)(prod_b >> 32), lo_b = (uint32_t)prod_b;
        uint32_t y0 = hi_b ^ x1 ^ k0;
        uint32_t y1 = lo_b;
        uint32_t y2 = hi_a ^ x3 ^ k1;
        uint32_t y3 = lo_a;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Bulk words for ids id0 .. id0+n_ids-1 at counter (step, id_lo, id_hi, tag); out is [n_ids][4]. */
void om_philox_words(uint64_t seed, uint64_t id0, uint64_t n_ids, uint32_t step, uint32_t tag, uint32_t* out)
{
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    for (uint64_t i = 0; i < n_ids; ++i) {
        uint64_t id = id0 + i;
        uint32_t ctr[4] = { step, (uint32_t)id, (uint32_t)(id >> 32), tag };
        om_philox(ctr, key, out + 4 * i);
    }
}
