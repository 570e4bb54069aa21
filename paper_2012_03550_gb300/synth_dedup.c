/*
 * Helper of the synthetic-input generator (synth.py): keep the first
 * occurrence of each key in draw order, i.e. sequential rejection of repeated
 * coordinates.  An open-addressing hash set (linear probing) holds the keys
 * accepted so far; it persists across calls so that rounds of draws can be
 * appended.  Holds no SGD_Tucker arithmetic.
 */
#include <stdint.h>

static inline uint64_t mix(uint64_t z)
{
    z ^= z >> 33;
    z *= 0xff51afd7ed558ccdULL;
    z ^= z >> 33;
    z *= 0xc4ceb9fe1a85ec53ULL;
    z ^= z >> 33;
    return z;
}

/* keys[n] (>= 0) in draw order; table[cap] zero-initialised by the caller
 * (cap a power of two, larger than twice the keys ever accepted).  Appends the
 * positions of newly seen keys to out (at most `need`) and returns how many
 * were appended. */
int64_t synth_first_unique(const int64_t *keys, int64_t n, int64_t need, int64_t *out,
                           uint64_t *table, int64_t cap)
{
    const uint64_t mask = (uint64_t)cap - 1;
    int64_t got = 0;
    for (int64_t i = 0; i < n && got < need; ++i) {
        const uint64_t k = (uint64_t)keys[i] + 1;   /* 0 marks an empty slot */
        uint64_t h = mix(k) & mask;
        for (;;) {
            const uint64_t t = table[h];
            if (t == 0) {
                table[h] = k;
                out[got++] = i;
                break;
            }
            if (t == k) break;
            h = (h + 1) & mask;
        }
    }
    return got;
}
