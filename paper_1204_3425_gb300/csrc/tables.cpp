// Host side of hubbard_sector_create: per-spin basis, ranking and hopping
// tables (Sec. 2.1 and the Kronecker split of Sec. 4.2).
#include <algorithm>
#include <cstdint>
#include <vector>

#include "internal.h"

namespace hub {

namespace {

// Binomial coefficients C(n, k) for n, k <= 32 (exact in uint64).
struct Binom {
    uint64_t c[33][33];
    Binom() {
        for (int n = 0; n <= 32; ++n) {
            c[n][0] = 1;
            for (int k = 1; k <= 32; ++k) c[n][k] = (k > n) ? 0 : (n == k ? 1 : c[n - 1][k - 1] + c[n - 1][k]);
        }
    }
};
const Binom& binom() {
    static Binom b;
    return b;
}

// Next larger word with the same popcount (Gosper's hack).
inline uint64_t next_same_popcount(uint64_t x) {
    uint64_t c = x & (~x + 1);
    uint64_t r = x + c;
    return (((r ^ x) >> 2) / c) | r;
}

// Position of `s` in the ascending list of words with popcount(s) bits set:
// the combinatorial number system, sum over set bits p_0 < p_1 < ... of
// C(p_k, k+1).  For a fixed popcount, ascending numeric order is colex order
// of the occupied-site sets, whose rank this is.
inline int64_t colex_rank(uint32_t s) {
    const Binom& B = binom();
    int64_t r = 0;
    int k = 0;
    while (s) {
        int p = __builtin_ctz(s);
        r += (int64_t)B.c[p][k + 1];
        ++k;
        s &= s - 1;
    }
    return r;
}

}  // namespace

void build_spin_tables(int ns, int n, const std::vector<std::pair<int, int>>& bonds, SpinTables& T) {
    T.ns = ns;
    T.n = n;
    T.D = (int64_t)binom().c[ns][n];
    T.states.resize((size_t)T.D);
    // ascending enumeration (Eq. J-formula)
    uint64_t w = (n == 0) ? 0 : ((n == 64) ? ~0ull : ((1ull << n) - 1));
    for (int64_t r = 0; r < T.D; ++r) {
        T.states[(size_t)r] = (uint32_t)w;
        if (n > 0 && r + 1 < T.D) w = next_same_popcount(w);
    }
    // hopping table: row r lists (r', sign) with <r'|H_sigma|r> = -t*sign (Sec. 2.1)
    T.rowptr.assign((size_t)T.D + 1, 0);
    T.tgt.clear();
    T.sign.clear();
    T.W = 0;
    std::vector<std::pair<int32_t, int8_t>> row;
    for (int64_t r = 0; r < T.D; ++r) {
        const uint32_t s = T.states[(size_t)r];
        row.clear();
        for (const auto& b : bonds) {
            const int i = b.first, j = b.second;
            const uint32_t bi = (s >> i) & 1u, bj = (s >> j) & 1u;
            if (bi == bj) continue;                   // both empty or both occupied
            const int lo = std::min(i, j), hi = std::max(i, j);
            // same-spin electrons on the sites strictly between the two ends
            const uint32_t between = (hi - lo > 1) ? (((1u << hi) - 1u) & ~((1u << (lo + 1)) - 1u)) : 0u;
            const int crossed = __builtin_popcount(s & between);
            const uint32_t s2 = s ^ (1u << i) ^ (1u << j);
            row.emplace_back((int32_t)colex_rank(s2), (int8_t)((crossed & 1) ? -1 : 1));
        }
        std::sort(row.begin(), row.end());
        for (const auto& e : row) {
            T.tgt.push_back(e.first);
            T.sign.push_back(e.second);
        }
        T.rowptr[(size_t)r + 1] = (int32_t)T.tgt.size();
        T.W = std::max<int>(T.W, (int)row.size());
    }
}

}  // namespace hub
