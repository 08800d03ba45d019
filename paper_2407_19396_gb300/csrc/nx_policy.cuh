// nx_policy.cuh -- the policy of the fused policy + environment rollout on
// the fifth-generation tensor cores (tcgen05, tensor memory).
//
// The policy (reading P1) maps each env's categorical first-person view (49
// entity codes, the input row x, padded to K = 64) through two hidden layers
// of 64 units to one logit per action:
//   h1 = clamp((W1 x + b1) >> shift1, 0, 255), h2 = clamp((W2 h1 + b2) >> shift2, 0, 255),
//   z = W3 h2 + b3,   greedy action = the first largest z over the family's actions.
// Weights are int8 and activations at most 255, so every product and every
// partial sum is an integer below 2^24: bf16 operands with fp32 accumulation
// give the exact integer result in any order of summation, and the tensor-core
// result equals the integer arithmetic bit for bit.
//
// One block holds 128 envs, one per thread and one per row of the tensor-core
// tile (M = 128) and of tensor memory (lane = row).  Per layer: every thread
// writes its row of the A operand (bf16, shared memory), one thread issues
// four tcgen05.mma (K = 16 each) against the layer's weights (the B operand,
// N x K) with the accumulator in tensor memory and commits them to an
// mbarrier; every thread waits (bounded), reads its row back with
// tcgen05.ld, requantises and writes the next layer's A row.  With fewer than
// 128 envs per weight set (16, 32 or 64) a block holds the images of its
// 8, 4 or 2 weight sets: each layer runs one MMA group per set over all 128
// rows into that set's own 64 tensor-memory columns (one commit), and each
// row reads the columns of its own set.
//
// Shared-memory operand layout (no swizzle, K-major): 8 x 16-byte core
// matrices; element (r, k) of a tile lives at
//   (r / 8) * 1024 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2,
// i.e. descriptor leading-dimension offset 128 bytes (the next core matrix
// along K) and stride offset 1024 bytes (the next 8 rows).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace nxp {

constexpr int kRows = 128;     // envs per block = M of every MMA
constexpr int kK = 64;         // inputs per layer (49 view cells + zero padding; 64 hidden units)
constexpr int kIn = 49;
constexpr int kATileBytes = kRows * kK * 2;  // 16 KB
// one agent's image of weights and biases in shared memory
constexpr int kW1 = 0, kW2 = 8192, kW3 = 16384;  // W1^T, W2^T: 64 x 64; W3^T: 16 x 64 (rows >= 7 zero)
// biases: layers 1 and 2 as f32 scaled by 2^-shift of their layer (exact:
// |b| <= 2^22), layer 3 as int32: 64, 64, 16
constexpr int kB1 = 18432, kB2 = 18688, kB3 = 18944;
constexpr int kImageBytes = 19008;
constexpr uint32_t kSbo = 1024, kLbo = 128;

__host__ __device__ constexpr uint32_t tile_offset(int r, int k)
{
    return (uint32_t)((r / 8) * kSbo + (k / 8) * kLbo + (r % 8) * 16 + (k % 8) * 2);
}

// instruction descriptor of kind::f16: f32 accumulator, bf16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

// shared-memory matrix descriptor: start address, leading / stride byte
// offsets (16-byte units), the fixed version bits 0b001 at bit 46, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(kLbo >> 4) << 16) | ((uint64_t)(kSbo >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// D[tmem] = A * B^T over K = 64 in four K = 16 steps (one thread)
__device__ __forceinline__ void mma_k64(uint32_t tmem, const uint8_t* sA, const uint8_t* sB, uint32_t idesc)
{
    const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
    for (int ks = 0; ks < kK / 16; ++ks) {
        const uint64_t ad = smem_desc(a0 + ks * 2 * kLbo), bd = smem_desc(b0 + ks * 2 * kLbo);
        const uint32_t acc = ks > 0 ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    }
}

__device__ __forceinline__ void mma_commit(uint64_t* mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
                 : "memory");
}

// Waits for the mbarrier phase with the given parity; gives up after a bounded
// number of polls and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity)
{
    uint32_t done = 0;
    for (int it = 0; it < (1 << 20) && !done; ++it) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(mbar)), "r"(parity)
            : "memory");
    }
    return done != 0;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// The threads' A rows (generic-proxy stores) and their tensor-memory reads
// are complete before the next MMA is issued.
__device__ __forceinline__ void sync_for_mma()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ uint32_t bf16_bits(int v) { return (uint32_t)__bfloat16_as_ushort(__int2bfloat16_rn(v)); }

// Writes 16 consecutive values of row r (k0 a multiple of 8) as bf16.
__device__ __forceinline__ void store_row16(uint8_t* sA, int r, int k0, const int (&x)[16])
{
    uint32_t w[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) w[j] = bf16_bits(x[2 * j]) | (bf16_bits(x[2 * j + 1]) << 16);
    *reinterpret_cast<uint4*>(sA + tile_offset(r, k0)) = make_uint4(w[0], w[1], w[2], w[3]);
    *reinterpret_cast<uint4*>(sA + tile_offset(r, k0 + 8)) = make_uint4(w[4], w[5], w[6], w[7]);
}

// The input row: the categorical first-person view (the entity byte of each
// of the 49 cells of the 147-byte symbolic record held as 37 stream words),
// zero beyond.
__device__ __forceinline__ void store_obs_row(uint8_t* sA, int r, const uint32_t (&sw)[37])
{
#pragma unroll
    for (int k0 = 0; k0 < kK; k0 += 16) {
        int x[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int c = k0 + j;
            x[j] = c < kIn ? (int)((sw[(3 * c) >> 2] >> (8 * ((3 * c) & 3))) & 0xFFu) : 0;
        }
        store_row16(sA, r, k0, x);
    }
}

__device__ __forceinline__ void store_zero_row(uint8_t* sA, int r)
{
#pragma unroll
    for (int k0 = 0; k0 < kK; k0 += 8) *reinterpret_cast<uint4*>(sA + tile_offset(r, k0)) = make_uint4(0, 0, 0, 0);
}

// Requantises 16 accumulators of this thread's row into bf16 activations:
// clamp(floor((acc + b) / 2^sh), 0, 255) in f32, exact since acc + b is an
// integer below 2^24 and the scaling is by a power of two.
// floor((acc + b) 2^-shift) as one fused multiply-add of the accumulator
// with the pre-scaled bias bs = b 2^-shift: |acc + b| < 2^23, so the product,
// the sum and hence the result are exact.
__device__ __forceinline__ void requant_row16(uint8_t* sA, int r, int k0, const uint32_t (&v)[16], const float* bs,
                                              float scale)
{
    uint32_t w[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float h0 = floorf(__fmaf_rn(__uint_as_float(v[2 * j]), scale, bs[2 * j]));
        float h1 = floorf(__fmaf_rn(__uint_as_float(v[2 * j + 1]), scale, bs[2 * j + 1]));
        h0 = fminf(fmaxf(h0, 0.0f), 255.0f);
        h1 = fminf(fmaxf(h1, 0.0f), 255.0f);
        const __nv_bfloat162 p2 = __floats2bfloat162_rn(h0, h1);  // low half: h0
        w[j] = *reinterpret_cast<const uint32_t*>(&p2);
    }
    *reinterpret_cast<uint4*>(sA + tile_offset(r, k0)) = make_uint4(w[0], w[1], w[2], w[3]);
    *reinterpret_cast<uint4*>(sA + tile_offset(r, k0 + 8)) = make_uint4(w[4], w[5], w[6], w[7]);
}

// 2^-sh as an f32 (sh in 0..24)
__device__ __forceinline__ float pow2_neg(int sh) { return __int_as_float((127 - sh) << 23); }

// All 128 threads of the block: after every thread wrote its input row, the
// first layer's MMA is issued (it then runs while the block does other work).
// MULTI: the block may hold several weight sets (`agents`), else one.
template <bool MULTI>
__device__ __forceinline__ void policy_issue_first(uint8_t* sA, const uint8_t* sW, uint32_t tmem, uint64_t* mbar,
                                                   int agents)
{
    sync_for_mma();
    if (threadIdx.x == 0) {
        if constexpr (MULTI) {
            for (int a = 0; a < agents; ++a)
                mma_k64(tmem + 64u * a, sA, sW + a * kImageBytes + kW1, idesc_bf16(kRows, kK));
        } else {
            mma_k64(tmem, sA, sW + kW1, idesc_bf16(kRows, kK));
        }
        mma_commit(mbar);
    }
}

// The weight sets of a block's rows (computed once per work item): the
// block's sets, this row's set, and the sets of this warp's rows (first, and
// one or two of them) -- each below 128 / envs_per_agent, so inside the
// allocated tensor-memory columns.
struct PolRows {
    int agents, mine, first, per_warp;
};
__device__ __forceinline__ PolRows pol_rows(int agents, int epa)
{
    const int tid = threadIdx.x, warp = tid >> 5;
    if (epa >= kRows) return PolRows{1, 0, 0, 1};
    return PolRows{agents, tid / epa, (32 * warp) / epa, epa < 32 ? 32 / epa : 1};
}

template <bool MULTI>
__device__ __forceinline__ int policy_finish(uint8_t* sA, const uint8_t* sW, uint32_t tmem, uint64_t* mbar,
                                             uint32_t& phase, int n_act, int shift1, int shift2, bool& ok,
                                             const PolRows& pr)
{
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);  // this warp's 32 lanes
    // (one weight set: the constants of pol_rows for envs_per_agent >= 128)
    const int agents = MULTI ? pr.agents : 1, mine = MULTI ? pr.mine : 0, first = MULTI ? pr.first : 0,
              per_warp = MULTI ? pr.per_warp : 1;
    const uint8_t* myW = sW + mine * kImageBytes;
#pragma unroll 1
    for (int layer = 0; layer < 2; ++layer) {
        if (layer == 1) {
            sync_for_mma();
            if (tid == 0) {
                for (int a = 0; a < agents; ++a)
                    mma_k64(tmem + 64u * a, sA, sW + a * kImageBytes + kW2, idesc_bf16(kRows, kK));
                mma_commit(mbar);
            }
        }
        ok = mbar_wait(mbar, phase) && ok;
        phase ^= 1u;
        __syncwarp();  // tcgen05.ld is warp-collective: converge after the per-thread wait
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const float* bs = reinterpret_cast<const float*>(myW + (layer ? kB2 : kB1));
        const float scale = pow2_neg(layer ? shift2 : shift1);
        if (per_warp == 1) {
            // every row of the warp has the warp's set
            const uint32_t tcol = trow + 64u * (uint32_t)first;
#pragma unroll 1
            for (int c0 = 0; c0 < kK; c0 += 16) {
                uint32_t v[16];
                tmem_ld16(tcol + (uint32_t)c0, v);
                requant_row16(sA, tid, c0, v, bs + c0, scale);
            }
        } else {
#pragma unroll 1
            for (int c0 = 0; c0 < kK; c0 += 16) {
#pragma unroll 1
                for (int j = 0; j < per_warp; ++j) {
                    uint32_t v[16];
                    tmem_ld16(trow + 64u * (uint32_t)(first + j) + (uint32_t)c0, v);
                    if (mine == first + j) requant_row16(sA, tid, c0, v, bs + c0, scale);
                }
            }
        }
    }
    sync_for_mma();
    if (tid == 0) {
        for (int a = 0; a < agents; ++a) mma_k64(tmem + 64u * a, sA, sW + a * kImageBytes + kW3, idesc_bf16(kRows, 16));
        mma_commit(mbar);
    }
    ok = mbar_wait(mbar, phase) && ok;
    phase ^= 1u;
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    uint32_t v[16] = {};
    if (per_warp == 1) {
        tmem_ld16(trow + 64u * (uint32_t)first, v);
    } else {
#pragma unroll 1
        for (int j = 0; j < per_warp; ++j) {
            uint32_t w[16];
            tmem_ld16(trow + 64u * (uint32_t)(first + j), w);
            if (mine == first + j) {
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = w[i];
            }
        }
    }
    const int32_t* b3 = reinterpret_cast<const int32_t*>(myW + kB3);
    int best = 0, bz = __float2int_rn(__uint_as_float(v[0])) + b3[0];
#pragma unroll
    for (int a = 1; a < 7; ++a) {
        const int z = __float2int_rn(__uint_as_float(v[a])) + b3[a];
        if (a < n_act && z > bz) {
            best = a;
            bz = z;
        }
    }
    return best;
}

}  // namespace nxp
