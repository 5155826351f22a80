// Building blocks of the tensor-core kernels (tcgen05): BF16 splitting,
// the K-major no-swizzle operand layout, bulk copies completed on an
// mbarrier, bounded mbarrier waits, shared-memory matrix descriptors, and the
// MMA / commit instructions.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace snn {
namespace tc {

constexpr int kRows = 128;            // rows (M or N) of one operand tile

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Element offset of (row, k) in the tiled K-major layout: tiles of 128 rows x
// tk K-elements, `kt` K tiles per 128-row band; inside a tile, core matrices
// of 8 rows x 8 BF16 (16 bytes), tk / 8 of them along K per 8-row group, so
// a tile is one contiguous block of 128 * tk elements.
__host__ __device__ __forceinline__ int64_t tiled_offset(int64_t row, int64_t k, int64_t kt, int tk) {
    const int64_t tile = (row / kRows) * kt + k / tk;
    const int r = (int)(row % kRows), c = (int)(k % tk);
    return tile * kRows * tk + ((r >> 3) * (tk / 8) + (c >> 3)) * 64 + (r & 7) * 8 + (c & 7);
}

__device__ __forceinline__ uint16_t bf16_rn(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }

__device__ __forceinline__ float bf16_to_f(uint16_t h) { return __bfloat162float(__ushort_as_bfloat16(h)); }

// x = hi + mid + lo (+ a remainder below FP32 resolution): each part the BF16
// rounding of what the previous parts left.
__device__ __forceinline__ void split3(float x, uint16_t& hi, uint16_t& mid, uint16_t& lo) {
    hi = bf16_rn(x);
    const float r1 = x - bf16_to_f(hi);
    mid = bf16_rn(r1);
    lo = bf16_rn(r1 - bf16_to_f(mid));
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    return done != 0;
}

// Bounded wait for phase `parity` of an mbarrier: false after `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t limit) {
    for (uint32_t it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

// Shared-memory matrix descriptor, K-major, no swizzle: start address, the
// byte distance between core matrices along K (leading) and along M/N
// (stride), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16 with an FP32 accumulator and BF16 A and
// B, both K-major, for an M x N tile.
constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// D (tensor memory) = A B^T (+ D when accumulate != 0), K = 16.
__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate) : "memory");
}

// Arrives on the mbarrier when every MMA issued so far by this thread is done.
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 32 consecutive FP32 columns of this warp's 32 tensor-memory lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
          "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
          "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
          "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ---- epilogue: a 128 x 128 FP32 accumulator into a row-major global matrix --
// Tensor memory gives each thread one row (lane) of the accumulator; adding
// that straight into global memory makes every warp-wide access touch 32
// rows.  Instead the tile goes through shared memory: the CTA's eight warps
// write it there row by row (phase 1), then each warp adds whole rows, lanes
// along the row, so global reads and writes are contiguous (phase 2).
constexpr int kTileLd = 132;          // padded row stride (floats): conflict-free float4 phases

// Phase 1, by all eight warps of the CTA: warp w reads lanes 32 (w % 4) .. + 31
// and columns 64 (w / 4) .. + 63 of the accumulator at column `tmem_col`.
__device__ __forceinline__ void tmem_tile_to_smem(uint32_t tmem_col, float* s, int warp, int lane) {
    const int q = warp & 3, h = warp >> 2;
    const int r = q * 32 + lane;
    for (int c0 = h * 64; c0 < h * 64 + 64; c0 += 32) {
        uint32_t v[32];
        tmem_ld32(tmem_col + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
        for (int k = 0; k < 32; k += 4)
            *reinterpret_cast<float4*>(s + r * kTileLd + c0 + k) =
                make_float4(__uint_as_float(v[k]), __uint_as_float(v[k + 1]), __uint_as_float(v[k + 2]),
                            __uint_as_float(v[k + 3]));
    }
}

// Phase 2, by all eight warps after a CTA barrier: D[r][c] += scale_r s[r][c]
// for r < rows, c < cols (D already offset to the tile's first element,
// row_scale to the tile's first row or nullptr for 1).  vec: 16-byte
// accesses (D 16-byte aligned, ldd a multiple of 4); kAtomic: atomic adds.
// A warp takes rows warp, warp + 8, ..., eight at a time, and loads all eight
// before it stores any, so eight row reads are in flight per warp.
template <bool kAtomic>
__device__ __forceinline__ void smem_tile_to_global(const float* s, float* D, int64_t ldd, int rows, int cols,
                                                    const float* row_scale, bool vec, int warp, int lane) {
    const bool full = vec && cols == 128;
    for (int r0 = warp; r0 < rows; r0 += 64) {
        if (full) {
            float4 o[8];
            if constexpr (!kAtomic) {
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int r = r0 + 8 * u;
                    if (r < rows) o[u] = *reinterpret_cast<const float4*>(D + (int64_t)r * ldd + 4 * lane);
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int r = r0 + 8 * u;
                if (r >= rows) continue;
                const float sc = row_scale ? row_scale[r] : 1.0f;
                const float4 a = *reinterpret_cast<const float4*>(s + r * kTileLd + 4 * lane);
                const float4 add = make_float4(sc * a.x, sc * a.y, sc * a.z, sc * a.w);
                float4* p = reinterpret_cast<float4*>(D + (int64_t)r * ldd + 4 * lane);
                if constexpr (kAtomic) {
                    atomicAdd(p, add);
                } else {
                    o[u].x += add.x; o[u].y += add.y; o[u].z += add.z; o[u].w += add.w;
                    *p = o[u];
                }
            }
        } else {
            // ragged or unaligned tile: four columns lane + 32 k per lane and row
            float o[8][4];
            if constexpr (!kAtomic) {
#pragma unroll
                for (int u = 0; u < 8; ++u)
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int r = r0 + 8 * u, c = lane + 32 * k;
                        if (r < rows && c < cols) o[u][k] = D[(int64_t)r * ldd + c];
                    }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int r = r0 + 8 * u;
                if (r >= rows) continue;
                const float sc = row_scale ? row_scale[r] : 1.0f;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int c = lane + 32 * k;
                    if (c >= cols) continue;
                    const float add = sc * s[r * kTileLd + c];
                    if constexpr (kAtomic) atomicAdd(D + (int64_t)r * ldd + c, add);
                    else D[(int64_t)r * ldd + c] = o[u][k] + add;
                }
            }
        }
    }
}

}  // namespace tc
}  // namespace snn
