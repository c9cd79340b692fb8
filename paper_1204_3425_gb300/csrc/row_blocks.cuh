// Device side of the row-phase hop table (SELL-32/8 with coloured slots):
// entry decoding and the per-lane walk over a group's slot blocks.  Shared by
// the single-sector row phase and the batched solver's row pass.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hub {

// row-phase entry: slot index in the low bits, top bit (15 or 31) = sign -1
template <typename EntT> struct RowEnt;
template <> struct RowEnt<uint16_t> {
    static __device__ __forceinline__ uint32_t idx(uint32_t e) { return e & 0x7FFFu; }
    static __device__ __forceinline__ int sgn(uint32_t e) { return ((int)(e << 16) >> 31) | 1; }
};
template <> struct RowEnt<uint32_t> {
    static __device__ __forceinline__ uint32_t idx(uint32_t e) { return e & 0x7FFFFFFFu; }
    static __device__ __forceinline__ int sgn(uint32_t e) { return ((int)e >> 31) | 1; }
};
// staged slots: D rounded up to 32, then 32 zero slots for padding entries
__host__ __device__ __forceinline__ int64_t staged_slots(int64_t D) { return (D + 31) / 32 * 32 + 32; }

// Hop sums of one lane over its group's slots (warp-sliced table): nhalf
// half-blocks of 4 slots per lane, stored as nhalf / 2 blocks of 8 slots
// ((b * 32 + lane) * 8 entries in) and, when nhalf is odd, one trailing
// block of 4 (at nblk * 256 + lane * 4).  Blocks are read with 16-byte loads,
// all blocks of a chunk before any gather, so one table-load latency is paid
// per chunk rather than per hop.  add(e) receives each entry.
template <typename EntT, typename F>
__device__ __forceinline__ void for_each_hop(const EntT* __restrict__ base, int nhalf, int lane, F&& add) {
    constexpr int LOADS = (int)sizeof(EntT);          // 16-byte loads per 8-slot block: 2 (u16) -> 1, 4 (u32) -> 2
    constexpr int NL = LOADS == 2 ? 1 : 2;
    constexpr int CH = NL == 1 ? 4 : 2;               // blocks per chunk
    const int nblk = nhalf >> 1;
    const uint4* p = reinterpret_cast<const uint4*>(base) + (int64_t)lane * NL;
    for (int b0 = 0; b0 < nblk; b0 += CH) {
        uint4 buf[CH][NL];
#pragma unroll
        for (int i = 0; i < CH; ++i)
#pragma unroll
            for (int j = 0; j < NL; ++j)
                buf[i][j] = (b0 + i < nblk) ? __ldg(p + (int64_t)(b0 + i) * 32 * NL + j) : make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int i = 0; i < CH; ++i) {
            if (b0 + i >= nblk) break;
#pragma unroll
            for (int j = 0; j < NL; ++j) {
                const uint32_t q[4] = {buf[i][j].x, buf[i][j].y, buf[i][j].z, buf[i][j].w};
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    if constexpr (NL == 1) {
                        add(q[r] & 0xFFFFu);
                        add(q[r] >> 16);
                    } else {
                        add(q[r]);
                    }
                }
            }
        }
    }
    if (nhalf & 1) {
        const EntT* h = base + (int64_t)nblk * 256;
        if constexpr (NL == 1) {
            const uint2 q = __ldg(reinterpret_cast<const uint2*>(h) + lane);
            add(q.x & 0xFFFFu);
            add(q.x >> 16);
            add(q.y & 0xFFFFu);
            add(q.y >> 16);
        } else {
            const uint4 q = __ldg(reinterpret_cast<const uint4*>(h) + lane);
            add(q.x);
            add(q.y);
            add(q.z);
            add(q.w);
        }
    }
}

}  // namespace hub
