// lev.cuh -- edit distance (unit costs) by the bit-parallel recurrence of
// Myers (1999) in the form for global distance (Hyyrö 2001: the top row of the
// dynamic-programming table grows by one per text character, so a 1 is
// shifted into the horizontal positive-delta vector).  The pattern occupies
// W 64-bit words; words above ceil(m/64) are skipped.
//
// lev_myers returns the distance when it is <= k and some value > k
// otherwise; it stops early once the bottom-row value can no longer fall to k.
#pragma once

#include <stdint.h>

#ifndef CT_HD
#define CT_HD __host__ __device__ __forceinline__
#endif

namespace ct {

inline int lev_words_for(int max_len) {
    int w = (max_len + 63) / 64;
    if (w <= 1) return 1;
    if (w <= 2) return 2;
    if (w <= 4) return 4;
    if (w <= 8) return 8;
    return 16;
}

// peq[c * W + w]: bit j set iff pattern[64 w + j] == c.
template <int W>
__device__ __forceinline__ void lev_build_peq(uint64_t *peq, const uint8_t *pat, int m) {
    for (int i = threadIdx.x; i < 256 * W; i += blockDim.x) peq[i] = 0ull;
    __syncthreads();
    for (int j = threadIdx.x; j < m; j += blockDim.x)
        atomicOr((unsigned long long *)&peq[pat[j] * W + (j >> 6)], 1ull << (j & 63));
}

template <int W>
CT_HD int lev_myers(const uint64_t *peq, int m, const uint8_t *txt, int n, int k) {
    if (k < 0) return 0 == m && 0 == n ? 0 : k + 1;
    int dl = m > n ? m - n : n - m;
    if (dl > k) return k + 1;
    if (m == 0) return n;
    if (n == 0) return m;
    const int nw = (m + 63) >> 6;
    const int hw = (m - 1) >> 6;
    const uint64_t hbit = 1ull << ((m - 1) & 63);
    uint64_t Pv[W], Mv[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
        Pv[w] = ~0ull;
        Mv[w] = 0ull;
    }
    int score = m;
    // the text is read a block of LEV_PF characters ahead of the recurrence:
    // independent loads, so that a step does not wait on its own load
    constexpr int LEV_PF = 8;
    int nxt[LEV_PF];
#pragma unroll
    for (int u = 0; u < LEV_PF; ++u) nxt[u] = u < n ? (int)txt[u] : 0;
    for (int j0 = 0; j0 < n; j0 += LEV_PF) {
        int blk[LEV_PF];
#pragma unroll
        for (int u = 0; u < LEV_PF; ++u) {
            blk[u] = nxt[u];
            nxt[u] = j0 + LEV_PF + u < n ? (int)txt[j0 + LEV_PF + u] : 0;
        }
#pragma unroll
        for (int u = 0; u < LEV_PF; ++u) {
            const int j = j0 + u;
            if (j >= n) break;
            const uint64_t *eqr = peq + blk[u] * W;
            uint64_t carry = 0ull, hp_in = 1ull, hn_in = 0ull;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                if (w < nw) {
                    uint64_t Eq = eqr[w];
                    uint64_t pv = Pv[w], mv = Mv[w];
                    uint64_t Xv = Eq | mv;
                    uint64_t t = Eq & pv;
                    uint64_t s1 = t + pv;
                    uint64_t c1 = s1 < t ? 1ull : 0ull;
                    uint64_t s2 = s1 + carry;
                    uint64_t c2 = s2 < s1 ? 1ull : 0ull;
                    carry = c1 | c2;
                    uint64_t Xh = (s2 ^ pv) | Eq;
                    uint64_t Ph = mv | ~(Xh | pv);
                    uint64_t Mh = pv & Xh;
                    if (w == hw) {
                        if (Ph & hbit) ++score;
                        else if (Mh & hbit) --score;
                    }
                    uint64_t ph_out = Ph >> 63, mh_out = Mh >> 63;
                    Ph = (Ph << 1) | hp_in;
                    Mh = (Mh << 1) | hn_in;
                    hp_in = ph_out;
                    hn_in = mh_out;
                    Pv[w] = Mh | ~(Xv | Ph);
                    Mv[w] = Ph & Xv;
                }
            }
            if (score - (n - 1 - j) > k) return k + 1;
        }
    }
    return score;
}

}  // namespace ct
