// Kernels of the learned surrogate: a 1-D convolutional operator over tubes
// that advances the macroscopic state (rho, u, T) by K lattice steps per call
// (the lbm_nn_* entry points of include/lbm.h).  The paper has no such
// network; it is an extension whose fallback, and the reference it is
// measured against, is the lattice Boltzmann method itself.
//
// Data layout (channel-last, one tube after another):
//   activations x[b][l][c] bfloat16, C channels (C a multiple of 128);
//   pre-activations z[b][l][c] bfloat16; residual-stream gradients gx fp32;
//   weights W[t][co][ci] bfloat16 (k taps, tap t reads position l + (t-k/2)d,
//   zero outside the tube), their transposed and flipped copy
//   WT[t][ci][co] = W[k-1-t][co][ci] for the input gradient.
//
// The three convolution products are implicit GEMMs on the fifth-generation
// tensor cores: the Tensor Memory Accelerator copies 128-byte-swizzled tiles
// straight out of the channel-last tensors (the tap shift is a coordinate
// offset; rows outside the tube come back as zeros), one thread issues
// tcgen05.mma into a 128 x 128 fp32 accumulator in tensor memory, and warps
// drain it with tcgen05.ld into a fused epilogue (4 warps in the
// one-tile-per-block form, 16 in the persistent form).
//   forward       D[pos][co] = sum_{t,ci} x[pos+s_t][ci] W[t][co][ci]   (A, B K-major)
//   input grad    D[pos][ci] = sum_{t,co} gz[pos+s_t][co] WT[t][ci][co] (A, B K-major)
//   weight grad   D[co][ci]  = sum_pos gz[pos][co] x[pos+s_t][ci]       (A, B MN-major)
// The forward and input-gradient products run persistent (impl 0: one block
// per SM, double-buffered accumulators so that the epilogue of a tile
// overlaps the MMAs of the next; impl 3: the same with channels x 256
// positions per tile and one activation window per channel chunk shared by
// the taps) or one tile per block (impl 2); a CUDA-core implementation of
// all three (impl 1) is the comparison point.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/lbm.h"

namespace {

// ---------------------------------------------------------------- constants
constexpr int kTile = 128;          // accumulator rows and columns
constexpr int kChunk = 64;          // bf16 elements in one 128-byte swizzle row
constexpr int kStages = 3;          // pipeline depth
constexpr int kStageBytes = 32768;  // A tile + B tile (16 KB each)
constexpr int kSmemBytes = kStages * kStageBytes + 1024 + 128;  // + alignment + barriers
constexpr int kWgRows = 64;         // positions per weight-gradient stage
constexpr long long kWaitCycles = 1ll << 32;  // bound on every mbarrier wait (~2 s)
constexpr int kTimeoutBit = 4;      // status bit set when a wait gives up

// ------------------------------------------------------------ math helpers
// tanh on the special-function unit (tanh.approx.f32: relative error about
// 2^-11, below the bfloat16 rounding the activations get next)
__device__ __forceinline__ float tanh_fast(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// GELU in its tanh form, x/2 (1 + tanh(c (x + 0.044715 x^3))), written as
// fma(x/2, tanh(u), x/2) with u = x (c + 0.044715 c x^2), and its derivative.
__device__ __forceinline__ float gelu(float x)
{
    const float c = 0.7978845608028654f;  // sqrt(2/pi)
    const float th = tanh_fast(x * fmaf(x * x, 0.044715f * c, c));
    const float h = 0.5f * x;
    return fmaf(h, th, h);
}

__device__ __forceinline__ float gelu_grad(float x)
{
    const float c = 0.7978845608028654f;
    const float th = tanh_fast(c * fmaf(0.044715f * x, x * x, x));
    return 0.5f * (1.0f + th) + 0.5f * x * (1.0f - th * th) * c * fmaf(3.0f * 0.044715f * x, x, 1.0f);
}

__device__ __forceinline__ void unpack8(const uint4 &q, float *v)
{
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&q);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 f = __bfloat1622float2(h[i]);
        v[2 * i] = f.x;
        v[2 * i + 1] = f.y;
    }
}

__device__ __forceinline__ uint4 pack8(const float *v)
{
    uint4 q;
    __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&q);
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    return q;
}

// ------------------------------------------------- barriers, TMA, tcgen05
__device__ __forceinline__ uint32_t saddr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}"
                 ::"r"(saddr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done) : "r"(saddr(bar)), "r"(parity) : "memory");
    return done != 0;
}

// Wait for the phase of `bar` with the given parity to complete; gives up
// after `budget` clock cycles (kWaitCycles by default), sets the timeout bit
// and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *status,
                                          long long budget = kWaitCycles)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > budget) {
            if (status) atomicOr(status, kTimeoutBit);
            return false;
        }
    }
    return true;
}

// Self-test of the bounded wait: one thread waits on a barrier that only it
// could complete (it arrives first when `arrive` is set); otherwise nothing
// arrives and the wait must give up after `budget` cycles.
__global__ void k_wait_selftest(long long budget, int arrive, int *status)
{
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(&bar)) : "memory");
    mbar_wait(&bar, 0, status, budget);
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x,
                                            int y)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3}], [%4];"
                 ::"r"(saddr(dst)), "l"(map), "r"(x), "r"(y), "r"(saddr(bar)) : "memory");
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x,
                                            int y, int z)
{
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4}], [%5];"
                 ::"r"(saddr(dst)), "l"(map), "r"(x), "r"(y), "r"(z), "r"(saddr(bar)) : "memory");
}

// Shared-memory matrix descriptor, 128-byte swizzle: start address, leading
// and stride byte offsets (16-byte units), descriptor version 1, layout 2.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= 1ull << 46;
    d |= 2ull << 61;
    return d;
}

// Instruction descriptor of kind::f16: fp32 accumulator, bf16 A and B,
// M = N = 128, operand majorness (0 = K-major, 1 = MN-major).
__host__ __device__ constexpr uint32_t instr_desc(uint32_t a_mn, uint32_t b_mn)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (a_mn << 15) | (b_mn << 16) |
           ((uint32_t)(kTile >> 3) << 17) | ((uint32_t)(kTile >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 ::"r"(tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate) : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(saddr(bar)) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 lanes x 32 consecutive fp32 columns of the accumulator.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
        "%30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    // the wait takes the registers as operands so that no use moves above it
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                   "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                   "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]),
                   "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
                   "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]),
                   "+r"(r[30]), "+r"(r[31])
                 :: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------ GEMM kernels
enum Epi : int { kEpiForward = 0, kEpiInputGrad = 1 };

struct ConvArgs {
    int B, L, C, k, dil;
    const __nv_bfloat16 *x;    // forward: residual input (= the A tensor)
    const float *bias;         // forward: [C]
    __nv_bfloat16 *y;          // forward: output
    __nv_bfloat16 *z;          // forward: pre-activation (may be null)
    float *gx;                 // input grad: residual-stream gradient, updated in place
    const __nv_bfloat16 *zprev;  // input grad: pre-activation of the layer below (may be null)
    __nv_bfloat16 *gzprev;     // input grad: its gradient, bf16(gx * gelu'(zprev))
    int *status;
};

// Epilogue of 32 consecutive accumulator columns c..c+31 of one position
// (element offset `base` of column 0 of the tile, output channel n0 + c).
template <int EPI>
__device__ __forceinline__ void epilogue32(const ConvArgs &a, const float (&v)[32], int64_t base,
                                           int n0, int c)
{
    if constexpr (EPI == kEpiForward) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float xr[8], yv[8], zv[8];
            unpack8(*reinterpret_cast<const uint4 *>(a.x + base + c + 8 * q), xr);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float zz = v[8 * q + j] + __ldg(a.bias + n0 + c + 8 * q + j);
                zv[j] = zz;
                yv[j] = xr[j] + gelu(zz);
            }
            *reinterpret_cast<uint4 *>(a.y + base + c + 8 * q) = pack8(yv);
            if (a.z) *reinterpret_cast<uint4 *>(a.z + base + c + 8 * q) = pack8(zv);
        }
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float g[8];
            float4 *gp = reinterpret_cast<float4 *>(a.gx + base + c + 8 * q);
            const float4 g0 = gp[0], g1 = gp[1];
            g[0] = g0.x + v[8 * q + 0]; g[1] = g0.y + v[8 * q + 1];
            g[2] = g0.z + v[8 * q + 2]; g[3] = g0.w + v[8 * q + 3];
            g[4] = g1.x + v[8 * q + 4]; g[5] = g1.y + v[8 * q + 5];
            g[6] = g1.z + v[8 * q + 6]; g[7] = g1.w + v[8 * q + 7];
            gp[0] = make_float4(g[0], g[1], g[2], g[3]);
            gp[1] = make_float4(g[4], g[5], g[6], g[7]);
            if (a.gzprev) {
                float zp[8], gz[8];
                unpack8(*reinterpret_cast<const uint4 *>(a.zprev + base + c + 8 * q), zp);
#pragma unroll
                for (int j = 0; j < 8; ++j) gz[j] = g[j] * gelu_grad(zp[j]);
                *reinterpret_cast<uint4 *>(a.gzprev + base + c + 8 * q) = pack8(gz);
            }
        }
    }
}

struct Smem {
    uint8_t *tiles;
    uint64_t *full, *empty, *done;
    uint32_t *tmem_slot;
};

__device__ __forceinline__ Smem carve(uint8_t *raw)
{
    Smem s;
    s.tiles = (uint8_t *)(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = (uint64_t *)(s.tiles + kStages * kStageBytes);
    s.full = bars;
    s.empty = bars + kStages;
    s.done = bars + 2 * kStages;
    s.tmem_slot = (uint32_t *)(bars + 2 * kStages + 1);
    return s;
}

__device__ __forceinline__ void setup(const Smem &s)
{
    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(&s.full[i], 1);
            mbar_init(&s.empty[i], 1);
        }
        mbar_init(s.done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(saddr(s.tmem_slot)), "r"(kTile) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

__device__ __forceinline__ void teardown(uint32_t tmem)
{
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTile)
                     : "memory");
    }
}

// Producer side shared by the kernels: after a failed wait, wait (bounded)
// for the loads already issued so that none lands after the block exits.
__device__ __forceinline__ void drain(const Smem &s, int issued, int *status)
{
    for (int kb = std::max(0, issued - kStages); kb < issued; ++kb)
        mbar_wait(&s.full[kb % kStages], (kb / kStages) & 1, status);
}

// Forward and input-gradient convolution: one 128-position x 128-channel
// output tile per block, K = k taps x C channels in 64-channel steps.
template <int EPI>
__global__ void __launch_bounds__(128, 1)
    k_conv_tc(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_w,
              ConvArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    const Smem s = carve(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int l0 = blockIdx.x * kTile, n0 = blockIdx.y * kTile, b = blockIdx.z;
    const int chunks = a.C / kChunk, nk = a.k * chunks;
    setup(s);
    const uint32_t tmem = *s.tmem_slot;
    __shared__ volatile int failed;
    if (threadIdx.x == 0) failed = 0;
    __syncthreads();

    if (warp == 0 && lane == 0) {  // TMA producer
        int kb = 0;
        for (; kb < nk; ++kb) {
            const int st = kb % kStages, use = kb / kStages;
            if (use > 0 && !mbar_wait(&s.empty[st], (use - 1) & 1, a.status)) {
                failed = 1;
                break;
            }
            const int t = kb / chunks, c0 = (kb % chunks) * kChunk;
            uint8_t *tile = s.tiles + st * kStageBytes;
            mbar_expect_tx(&s.full[st], kStageBytes);
            tma_load_3d(tile, &map_a, &s.full[st], c0, l0 + (t - a.k / 2) * a.dil, b);
            tma_load_2d(tile + kStageBytes / 2, &map_w, &s.full[st], c0, t * a.C + n0);
        }
        if (kb < nk) drain(s, kb, a.status);
    } else if (warp == 1 && lane == 0) {  // MMA issuer
        constexpr uint32_t idesc = instr_desc(0, 0);
        for (int kb = 0; kb < nk; ++kb) {
            const int st = kb % kStages;
            if (!mbar_wait(&s.full[st], (kb / kStages) & 1, a.status)) {
                failed = 1;
                break;
            }
            tc_fence_after();
            const uint32_t at = saddr(s.tiles + st * kStageBytes);
            const uint32_t bt = at + kStageBytes / 2;
#pragma unroll
            for (int kk = 0; kk < kChunk / 16; ++kk)
                mma_bf16(tmem, smem_desc(at + kk * 32, 16, 1024), smem_desc(bt + kk * 32, 16, 1024),
                         idesc, (kb | kk) != 0);
            mma_commit(&s.empty[st]);
        }
        mma_commit(s.done);
    }
    __syncwarp();
    if (!mbar_wait(s.done, 0, a.status)) failed = 1;
    __syncwarp();
    tc_fence_after();

    const int row = warp * 32 + lane, l = l0 + row;
    const bool ok = l < a.L;
    const int64_t base = ((int64_t)b * a.L + l) * a.C + n0;
#pragma unroll 1
    for (int c = 0; c < kTile; c += 32) {
        float v[32];
        __syncwarp();  // tcgen05.ld is warp-collective
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + c, v);
        if (!ok || failed) continue;
        epilogue32<EPI>(a, v, base, n0, c);
    }
    teardown(tmem);
}

// Persistent form of the forward / input-gradient product: one block per
// SM walks the output tiles (128 positions x 128 channels) with a stride of
// the grid.  Warp 0 issues the TMA loads into a 4-stage ring, warp 1 issues
// the MMAs into one of two 128-column accumulators in tensor memory, and 16
// epilogue warps drain the other accumulator (warps 2..17: lane quarter
// warp % 4, 32 columns each), so the epilogue of one tile overlaps the MMAs
// of the next.
constexpr int kPStages = 4;
constexpr int kEpiWarps = 16;    // 4 per lane quarter, 32 accumulator columns each
constexpr int kPThreads = 64 + 32 * kEpiWarps;
constexpr int kStagePitch = 36;  // floats per staged row (32 + 4: conflict-free float4 rows)
constexpr int kStagingBytes = kEpiWarps * 32 * kStagePitch * 4;
constexpr int kPSmemBytes = kPStages * kStageBytes + kStagingBytes + 1024 + 256;

// Epilogue of one warp's 32 rows x COLS columns (32 or 64) of a persistent
// tile.  The accumulator rows (one per lane after tcgen05.ld) are transposed
// through a padded shared-memory block (pitch COLS + 4 floats) so that every
// global load and store is done cooperatively: COLS/4 lanes cover the COLS
// columns of one row, so each instruction touches whole row segments.
template <int EPI, int COLS = 64>
__device__ __forceinline__ void finish_rows(const ConvArgs &a, const float *st, int b, int l_first,
                                            int n0, bool skip);

template <int EPI, int COLS = 64>
__device__ __forceinline__ void epilogue_rows(const ConvArgs &a, float *st, uint32_t taddr, int b,
                                              int l_first, int n0, bool skip)
{
    constexpr int kPitch = COLS + 4;
    const int lane = threadIdx.x & 31;
#pragma unroll 1
    for (int c = 0; c < COLS; c += 32) {
        float v[32];
        __syncwarp();
        tmem_ld32(taddr + c, v);
#pragma unroll
        for (int j = 0; j < 8; ++j)
            *reinterpret_cast<float4 *>(st + lane * kPitch + c + 4 * j) =
                make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
    }
    __syncwarp();
    finish_rows<EPI, COLS>(a, st, b, l_first, n0, skip);
}

// Second half of the epilogue: the staged block (32 rows = positions
// l_first.., COLS channels n0.., pitch COLS + 4 floats) is read back so
// that COLS/4 lanes cover the COLS channels of one row and every global
// load and store touches whole row segments.
template <int EPI, int COLS>
__device__ __forceinline__ void finish_rows(const ConvArgs &a, const float *st, int b, int l_first,
                                            int n0, bool skip)
{
    constexpr int kPitch = COLS + 4, kLpr = COLS / 4, kRpi = 32 / kLpr, kBatch = 4;
    const int lane = threadIdx.x & 31;
    if (!skip) {
        const int cg = (lane % kLpr) * 4;
        float4 bias = make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr (EPI == kEpiForward) bias = *reinterpret_cast<const float4 *>(a.bias + n0 + cg);
        // 32 / kRpi rows per lane (r = lane / kLpr + kRpi i) in groups of
        // kBatch: all loads of a group are issued before any result is formed
        const int64_t row0 = ((int64_t)b * a.L + l_first) * a.C + n0 + cg;
#pragma unroll 1
        for (int r0 = lane / kLpr; r0 < 32; r0 += kBatch * kRpi) {
            float4 acc[kBatch], gin[kBatch];
            uint2 in[kBatch];
            bool live[kBatch];
#pragma unroll
            for (int i = 0; i < kBatch; ++i) {
                const int r = r0 + kRpi * i, l = l_first + r;
                live[i] = l < a.L;
                acc[i] = *reinterpret_cast<const float4 *>(st + r * kPitch + cg);
                if (live[i]) {
                    const int64_t o = row0 + (int64_t)(r * a.C);
                    if constexpr (EPI == kEpiForward) {
                        in[i] = *reinterpret_cast<const uint2 *>(a.x + o);
                    } else {
                        gin[i] = *reinterpret_cast<const float4 *>(a.gx + o);
                        if (a.gzprev) in[i] = *reinterpret_cast<const uint2 *>(a.zprev + o);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < kBatch; ++i) {
                if (!live[i]) continue;
                const int64_t o = row0 + (int64_t)((r0 + kRpi * i) * a.C);
                if constexpr (EPI == kEpiForward) {
                    const float2 x01 =
                        __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&in[i].x));
                    const float2 x23 =
                        __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&in[i].y));
                    const float z0 = acc[i].x + bias.x, z1 = acc[i].y + bias.y,
                                z2 = acc[i].z + bias.z, z3 = acc[i].w + bias.w;
                    uint2 yv;
                    *reinterpret_cast<__nv_bfloat162 *>(&yv.x) =
                        __floats2bfloat162_rn(x01.x + gelu(z0), x01.y + gelu(z1));
                    *reinterpret_cast<__nv_bfloat162 *>(&yv.y) =
                        __floats2bfloat162_rn(x23.x + gelu(z2), x23.y + gelu(z3));
                    *reinterpret_cast<uint2 *>(a.y + o) = yv;
                    if (a.z) {
                        uint2 zv;
                        *reinterpret_cast<__nv_bfloat162 *>(&zv.x) = __floats2bfloat162_rn(z0, z1);
                        *reinterpret_cast<__nv_bfloat162 *>(&zv.y) = __floats2bfloat162_rn(z2, z3);
                        *reinterpret_cast<uint2 *>(a.z + o) = zv;
                    }
                } else {
                    float4 g = gin[i];
                    g.x += acc[i].x, g.y += acc[i].y, g.z += acc[i].z, g.w += acc[i].w;
                    *reinterpret_cast<float4 *>(a.gx + o) = g;
                    if (a.gzprev) {
                        const float2 z01 =
                            __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&in[i].x));
                        const float2 z23 =
                            __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&in[i].y));
                        uint2 gv;
                        *reinterpret_cast<__nv_bfloat162 *>(&gv.x) =
                            __floats2bfloat162_rn(g.x * gelu_grad(z01.x), g.y * gelu_grad(z01.y));
                        *reinterpret_cast<__nv_bfloat162 *>(&gv.y) =
                            __floats2bfloat162_rn(g.z * gelu_grad(z23.x), g.w * gelu_grad(z23.y));
                        *reinterpret_cast<uint2 *>(a.gzprev + o) = gv;
                    }
                }
            }
        }
    }
    __syncwarp();  // the staging block is rewritten by the next tile
}

template <int EPI>
__global__ void __launch_bounds__(kPThreads, 1)
    k_conv_tcp(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_w,
               ConvArgs a, int tiles_l, int tiles_n, int total)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *tiles = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    float *staging = (float *)(tiles + kPStages * kStageBytes);
    uint64_t *full = (uint64_t *)(tiles + kPStages * kStageBytes + kStagingBytes);
    uint64_t *empty = full + kPStages;
    uint64_t *tfull = empty + kPStages;   // accumulator a ready for the epilogue
    uint64_t *tempty = tfull + 2;         // accumulator a drained by the epilogue
    uint32_t *tmem_slot = (uint32_t *)(tempty + 2);
    __shared__ volatile int failed;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kPStages; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&tfull[i], 1);
            mbar_init(&tempty[i], kEpiWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        failed = 0;
    }
    __syncwarp();
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(saddr(tmem_slot)), "r"(2 * kTile) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int chunks = a.C / kChunk, nk = a.k * chunks;

    if (warp == 0) {
        if (lane == 0) {  // TMA producer
            int g = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < total && ok; tile += gridDim.x) {
                const int n0 = (tile % tiles_n) * kTile, rest = tile / tiles_n;
                const int b = rest / tiles_l, l0 = (rest % tiles_l) * kTile;
                for (int kb = 0; kb < nk; ++kb, ++g) {
                    const int st = g % kPStages, use = g / kPStages;
                    if (use > 0 && !mbar_wait(&empty[st], (use - 1) & 1, a.status)) {
                        failed = 1;
                        ok = false;
                        break;
                    }
                    const int t = kb / chunks, c0 = (kb % chunks) * kChunk;
                    uint8_t *buf = tiles + st * kStageBytes;
                    mbar_expect_tx(&full[st], kStageBytes);
                    tma_load_3d(buf, &map_a, &full[st], c0, l0 + (t - a.k / 2) * a.dil, b);
                    tma_load_2d(buf + kStageBytes / 2, &map_w, &full[st], c0, t * a.C + n0);
                }
            }
            // wait (bounded) for the last loads so that none lands after exit
            for (int q = std::max(0, g - kPStages); q < g; ++q)
                mbar_wait(&full[q % kPStages], (q / kPStages) & 1, a.status);
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            constexpr uint32_t idesc = instr_desc(0, 0);
            int g = 0, it = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < total && ok; tile += gridDim.x, ++it) {
                const int acc = it & 1, use = it >> 1;
                const uint32_t d = tmem + acc * kTile;
                if (use > 0 && !mbar_wait(&tempty[acc], (use - 1) & 1, a.status)) {
                    failed = 1;
                    break;
                }
                tc_fence_after();
                for (int kb = 0; kb < nk; ++kb, ++g) {
                    const int st = g % kPStages;
                    if (!mbar_wait(&full[st], (g / kPStages) & 1, a.status)) {
                        failed = 1;
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t at = saddr(tiles + st * kStageBytes);
                    const uint32_t bt = at + kStageBytes / 2;
#pragma unroll
                    for (int kk = 0; kk < kChunk / 16; ++kk)
                        mma_bf16(d, smem_desc(at + kk * 32, 16, 1024),
                                 smem_desc(bt + kk * 32, 16, 1024), idesc, (kb | kk) != 0);
                    mma_commit(&empty[st]);
                }
                mma_commit(&tfull[acc]);
            }
        }
    } else {  // epilogue warps
        const int e = warp - 2, quarter = warp & 3, col0 = (e >> 2) * 32;
        int it = 0;
        for (int tile = blockIdx.x; tile < total; tile += gridDim.x, ++it) {
            const int acc = it & 1, use = it >> 1;
            const int n0 = (tile % tiles_n) * kTile, rest = tile / tiles_n;
            const int b = rest / tiles_l, l0 = (rest % tiles_l) * kTile;
            bool ready = mbar_wait(&tfull[acc], use & 1, a.status);
            __syncwarp();
            if (!ready) failed = 1;
            tc_fence_after();
            epilogue_rows<EPI, 32>(a, staging + e * 32 * kStagePitch,
                                   tmem + acc * kTile + ((uint32_t)(quarter * 32) << 16) + col0, b,
                                   l0 + quarter * 32, n0 + col0, failed != 0);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(&tempty[acc]))
                                        : "memory");
            if (failed) break;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTile)
                     : "memory");
    }
}

// Persistent form with the roles of the operands exchanged (impl 3): the
// output channels are the MMA's M = 128 rows (A = the weight tile, K-major)
// and 256 positions its N columns (B = activations, K-major), so one
// tcgen05.mma of 128 x 256 x 16 reads 12 KB of operands from shared memory
// instead of 16 KB for the same work as two 128 x 128 x 16 ones.  For each
// 64-channel chunk one window of 256 + (k-1) dil positions is loaded once
// and the k taps read it at row offsets t dil (sub-window descriptors),
// instead of one shifted tile per tap; the weight tiles stream through a
// 4-stage ring.  Two 256-column accumulators fill the 512 columns of tensor
// memory.  After tcgen05.ld a lane holds one channel at 32 positions; the
// staging store writes it transposed, so the read-back and the global I/O
// are those of the other persistent form.
constexpr int kNPos = 256;                         // positions per tile (MMA N)
constexpr int kXStages = 2;                        // activation windows in flight
constexpr int kWStages = 4;                        // weight tiles in flight
constexpr int kWTileBytes = kTile * kChunk * 2;    // 128 channels x 64 input channels
constexpr int kMaxHalo = 64;                       // largest (k-1) dil a window holds
constexpr int kNSmemFixed = kWStages * kWTileBytes + kStagingBytes + 1024 + 256;

// Window rows: 256 + (k-1) dil rounded up to 16, loaded as two boxes of
// half that (each a multiple of 8 rows, so both halves start 1024-byte aligned).
__host__ __device__ constexpr int window_rows(int k, int dil)
{
    return kNPos + ((k - 1) * dil + 15) / 16 * 16;
}
__host__ __device__ constexpr int tcn_smem_bytes(int rows) { return kNSmemFixed + kXStages * rows * 128; }
constexpr int kNSmemMax = kNSmemFixed + kXStages * (kNPos + kMaxHalo) * 128;
static_assert(kNSmemMax <= 227 * 1024, "shared memory of the transposed persistent form");
static_assert((kNPos + kMaxHalo) / 2 <= 256, "TMA box rows");

// Instruction descriptor of kind::f16 with fp32 accumulation, bf16 operands,
// M x N, both operands K-major.
__host__ __device__ constexpr uint32_t instr_desc_mn(uint32_t m, uint32_t n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}

template <int EPI>
__global__ void __launch_bounds__(kPThreads, 1)
    k_conv_tcn(const __grid_constant__ CUtensorMap map_x, const __grid_constant__ CUtensorMap map_w,
               ConvArgs a, int tiles_l, int tiles_m, int total, int rows)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *wbuf = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *xbuf = wbuf + kWStages * kWTileBytes;
    const int xbytes = rows * 128;
    float *staging = (float *)(xbuf + kXStages * xbytes);
    uint64_t *wfull = (uint64_t *)((uint8_t *)staging + kStagingBytes);
    uint64_t *wempty = wfull + kWStages;
    uint64_t *xfull = wempty + kWStages;
    uint64_t *xempty = xfull + kXStages;
    uint64_t *tfull = xempty + kXStages;   // accumulator a ready for the epilogue
    uint64_t *tempty = tfull + 2;          // accumulator a drained by the epilogue
    uint32_t *tmem_slot = (uint32_t *)(tempty + 2);
    __shared__ volatile int failed;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kWStages; ++i) {
            mbar_init(&wfull[i], 1);
            mbar_init(&wempty[i], 1);
        }
        for (int i = 0; i < kXStages; ++i) {
            mbar_init(&xfull[i], 1);
            mbar_init(&xempty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&tfull[i], 1);
            mbar_init(&tempty[i], kEpiWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        failed = 0;
    }
    __syncwarp();
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(saddr(tmem_slot)), "r"(2 * kNPos) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int chunks = a.C / kChunk;
    const int halo = (a.k / 2) * a.dil;  // window row 0 is position l0 - halo

    if (warp == 0) {
        if (lane == 0) {  // TMA producer
            int gx = 0, gw = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < total && ok; tile += gridDim.x) {
                const int co0 = (tile % tiles_m) * kTile, rest = tile / tiles_m;
                const int b = rest / tiles_l, l0 = (rest % tiles_l) * kNPos;
                for (int ch = 0; ch < chunks && ok; ++ch, ++gx) {
                    const int xs = gx % kXStages, xuse = gx / kXStages;
                    if (xuse > 0 && !mbar_wait(&xempty[xs], (xuse - 1) & 1, a.status)) {
                        failed = 1;
                        ok = false;
                        break;
                    }
                    uint8_t *win = xbuf + xs * xbytes;
                    mbar_expect_tx(&xfull[xs], xbytes);
                    tma_load_3d(win, &map_x, &xfull[xs], ch * kChunk, l0 - halo, b);
                    tma_load_3d(win + xbytes / 2, &map_x, &xfull[xs], ch * kChunk,
                                l0 - halo + rows / 2, b);
                    for (int t = 0; t < a.k; ++t, ++gw) {
                        const int ws = gw % kWStages, wuse = gw / kWStages;
                        if (wuse > 0 && !mbar_wait(&wempty[ws], (wuse - 1) & 1, a.status)) {
                            failed = 1;
                            ok = false;
                            break;
                        }
                        mbar_expect_tx(&wfull[ws], kWTileBytes);
                        tma_load_2d(wbuf + ws * kWTileBytes, &map_w, &wfull[ws], ch * kChunk,
                                    t * a.C + co0);
                    }
                }
            }
            // wait (bounded) for the last loads so that none lands after exit
            for (int q = std::max(0, gx - kXStages); q < gx; ++q)
                mbar_wait(&xfull[q % kXStages], (q / kXStages) & 1, a.status);
            for (int q = std::max(0, gw - kWStages); q < gw; ++q)
                mbar_wait(&wfull[q % kWStages], (q / kWStages) & 1, a.status);
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            constexpr uint32_t idesc = instr_desc_mn(kTile, kNPos);
            int gx = 0, gw = 0, it = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < total && ok; tile += gridDim.x, ++it) {
                const int acc = it & 1, use = it >> 1;
                const uint32_t d = tmem + acc * kNPos;
                if (use > 0 && !mbar_wait(&tempty[acc], (use - 1) & 1, a.status)) {
                    failed = 1;
                    break;
                }
                tc_fence_after();
                for (int ch = 0; ch < chunks && ok; ++ch, ++gx) {
                    const int xs = gx % kXStages;
                    if (!mbar_wait(&xfull[xs], (gx / kXStages) & 1, a.status)) {
                        failed = 1;
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t xt = saddr(xbuf + xs * xbytes);
                    for (int t = 0; t < a.k; ++t, ++gw) {
                        const int ws = gw % kWStages;
                        if (!mbar_wait(&wfull[ws], (gw / kWStages) & 1, a.status)) {
                            failed = 1;
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t wt = saddr(wbuf + ws * kWTileBytes);
                        const uint32_t bt = xt + (uint32_t)(t * a.dil) * 128u;
#pragma unroll
                        for (int kk = 0; kk < kChunk / 16; ++kk)
                            mma_bf16(d, smem_desc(wt + kk * 32, 16, 1024),
                                     smem_desc(bt + kk * 32, 16, 1024), idesc, (ch | t | kk) != 0);
                        mma_commit(&wempty[ws]);
                    }
                    mma_commit(&xempty[xs]);
                }
                mma_commit(&tfull[acc]);
            }
        }
    } else {  // epilogue warps: lane quarter warp % 4 (32 channels), 64 positions each
        const int e = warp - 2, quarter = warp & 3, pos0 = (e >> 2) * 64;
        float *st = staging + e * 32 * kStagePitch;
        int it = 0;
        for (int tile = blockIdx.x; tile < total; tile += gridDim.x, ++it) {
            const int acc = it & 1, use = it >> 1;
            const int co0 = (tile % tiles_m) * kTile, rest = tile / tiles_m;
            const int b = rest / tiles_l, l0 = (rest % tiles_l) * kNPos;
            bool ready = mbar_wait(&tfull[acc], use & 1, a.status);
            __syncwarp();
            if (!ready) failed = 1;
            tc_fence_after();
#pragma unroll 1
            for (int h = 0; h < 64; h += 32) {
                float v[32];
                __syncwarp();
                tmem_ld32(tmem + acc * kNPos + ((uint32_t)(quarter * 32) << 16) + pos0 + h, v);
#pragma unroll
                for (int j = 0; j < 32; ++j) st[j * kStagePitch + lane] = v[j];
                __syncwarp();
                finish_rows<EPI, 32>(a, st, b, l0 + pos0 + h, co0 + quarter * 32, failed != 0);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(&tempty[acc]))
                                        : "memory");
            if (failed) break;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kNPos)
                     : "memory");
    }
}

// Weight gradient: one block reduces the positions of blocks [q0, q1) (64
// positions each, tubes one after another) for one tap and one 128 x 128
// (co, ci) tile, then adds its tile to gw with coalesced vector reductions.
__global__ void __launch_bounds__(128, 1)
    k_wgrad_tc(const __grid_constant__ CUtensorMap map_g, const __grid_constant__ CUtensorMap map_x,
               float *gw, int B, int L, int C, int k, int dil, int per_block, int *status)
{
    extern __shared__ uint8_t smem_raw[];
    const Smem s = carve(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles = C / kTile;
    const int t = blockIdx.y / (tiles * tiles);
    const int co0 = ((blockIdx.y / tiles) % tiles) * kTile, ci0 = (blockIdx.y % tiles) * kTile;
    const int nblk = (L + kWgRows - 1) / kWgRows;
    const int total = B * nblk;
    const int q0 = blockIdx.x * per_block, q1 = std::min(total, q0 + per_block);
    if (q0 >= q1) return;  // uniform across the block, before any allocation
    const int nk = q1 - q0, shift = (t - k / 2) * dil;
    setup(s);
    const uint32_t tmem = *s.tmem_slot;
    __shared__ volatile int failed;
    if (threadIdx.x == 0) failed = 0;
    __syncthreads();

    if (warp == 0 && lane == 0) {
        int kb = 0;
        for (; kb < nk; ++kb) {
            const int st = kb % kStages, use = kb / kStages;
            if (use > 0 && !mbar_wait(&s.empty[st], (use - 1) & 1, status)) {
                failed = 1;
                break;
            }
            const int q = q0 + kb, bb = q / nblk, lb = (q % nblk) * kWgRows;
            uint8_t *tile = s.tiles + st * kStageBytes;
            mbar_expect_tx(&s.full[st], kStageBytes);
            // A = gz rows lb..lb+63, channel blocks co0 and co0+64 (8 KB each)
            tma_load_3d(tile, &map_g, &s.full[st], co0, lb, bb);
            tma_load_3d(tile + 8192, &map_g, &s.full[st], co0 + kChunk, lb, bb);
            // B = x rows lb+shift.., channel blocks ci0 and ci0+64
            tma_load_3d(tile + 16384, &map_x, &s.full[st], ci0, lb + shift, bb);
            tma_load_3d(tile + 24576, &map_x, &s.full[st], ci0 + kChunk, lb + shift, bb);
        }
        if (kb < nk) drain(s, kb, status);
    } else if (warp == 1 && lane == 0) {
        constexpr uint32_t idesc = instr_desc(1, 1);
        for (int kb = 0; kb < nk; ++kb) {
            const int st = kb % kStages;
            if (!mbar_wait(&s.full[st], (kb / kStages) & 1, status)) {
                failed = 1;
                break;
            }
            tc_fence_after();
            const uint32_t at = saddr(s.tiles + st * kStageBytes);
            const uint32_t bt = at + kStageBytes / 2;
            // 16 positions = two 8-row swizzle atoms (2048 bytes) per MMA;
            // the two 64-channel blocks are 8192 bytes apart
#pragma unroll
            for (int kk = 0; kk < kWgRows / 16; ++kk)
                mma_bf16(tmem, smem_desc(at + kk * 2048, 8192, 1024),
                         smem_desc(bt + kk * 2048, 8192, 1024), idesc, (kb | kk) != 0);
            mma_commit(&s.empty[st]);
        }
        mma_commit(s.done);
    }
    __syncwarp();
    if (!mbar_wait(s.done, 0, status)) failed = 1;
    __syncwarp();
    tc_fence_after();

    // stage 32 x 32 blocks through shared memory (the pipeline buffers are
    // free once the last MMA has completed) so that a warp adds 32
    // consecutive columns of one row at a time
    float *stage = reinterpret_cast<float *>(s.tiles) + warp * 32 * 33;
#pragma unroll 1
    for (int c = 0; c < kTile; c += 32) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + c, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) stage[lane * 33 + j] = v[j];
        __syncwarp();
        if (!failed) {
            // lane handles 4 consecutive columns of rows r = lane/8 + 4i
            const int cc = (lane & 7) * 4;
#pragma unroll 1
            for (int r = lane >> 3; r < 32; r += 4) {
                const int co = co0 + warp * 32 + r;
                float *dst = gw + ((int64_t)t * C + co) * C + ci0 + c + cc;
                const float *src = stage + r * 33 + cc;
                asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};"
                             ::"l"(dst), "f"(src[0]), "f"(src[1]), "f"(src[2]), "f"(src[3])
                             : "memory");
            }
        }
        __syncwarp();
    }
    teardown(tmem);
}

// ------------------------------------------------- CUDA-core comparison path
constexpr int kSimtTX = 128, kSimtTC = 64, kSimtCI = 32, kSimtMaxK = 7;
constexpr int kSimtMaxSpan = kSimtTX + (kSimtMaxK - 1) * 16;

// out tile [128 positions][64 channels] of sum_t in[pos + s_t][ci] w[t][n][ci]
__device__ __forceinline__ void simt_tile(const __nv_bfloat16 *in, const __nv_bfloat16 *w, int L,
                                          int C, int k, int dil, int b, int x0, int n0,
                                          float (&acc)[8][4])
{
    __shared__ float xs[kSimtMaxSpan][kSimtCI + 1];
    __shared__ float ws[kSimtTC][kSimtMaxK][kSimtCI + 1];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int half = k / 2, span = kSimtTX + (k - 1) * dil;
    for (int ci0 = 0; ci0 < C; ci0 += kSimtCI) {
        for (int e = tid; e < span * kSimtCI; e += 256) {
            const int r = e / kSimtCI, c = e % kSimtCI, l = x0 - half * dil + r;
            xs[r][c] = (l >= 0 && l < L) ? __bfloat162float(in[((int64_t)b * L + l) * C + ci0 + c]) : 0.f;
        }
        for (int e = tid; e < kSimtTC * k * kSimtCI; e += 256) {
            const int c = e % kSimtCI, t = (e / kSimtCI) % k, o = e / (kSimtCI * k);
            ws[o][t][c] = __bfloat162float(w[((int64_t)t * C + n0 + o) * C + ci0 + c]);
        }
        __syncthreads();
        for (int t = 0; t < k; ++t) {
#pragma unroll 4
            for (int c = 0; c < kSimtCI; ++c) {
                float wv[4], xv[8];
#pragma unroll
                for (int j = 0; j < 4; ++j) wv[j] = ws[tx * 4 + j][t][c];
#pragma unroll
                for (int i = 0; i < 8; ++i) xv[i] = xs[ty * 8 + i + t * dil][c];
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(xv[i], wv[j], acc[i][j]);
            }
        }
        __syncthreads();
    }
}

template <int EPI>
__global__ void __launch_bounds__(256) k_conv_simt(const __nv_bfloat16 *in, const __nv_bfloat16 *w,
                                                   ConvArgs a)
{
    const int x0 = blockIdx.x * kSimtTX, n0 = blockIdx.y * kSimtTC, b = blockIdx.z;
    float acc[8][4] = {};
    simt_tile(in, w, a.L, a.C, a.k, a.dil, b, x0, n0, acc);
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int l = x0 + ty * 8 + i;
        if (l >= a.L) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            const int64_t o = ((int64_t)b * a.L + l) * a.C + n;
            if constexpr (EPI == kEpiForward) {
                const float zz = acc[i][j] + a.bias[n];
                a.y[o] = __float2bfloat16_rn(__bfloat162float(a.x[o]) + gelu(zz));
                if (a.z) a.z[o] = __float2bfloat16_rn(zz);
            } else {
                const float g = a.gx[o] + acc[i][j];
                a.gx[o] = g;
                if (a.gzprev) a.gzprev[o] = __float2bfloat16_rn(g * gelu_grad(__bfloat162float(a.zprev[o])));
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_wgrad_simt(const __nv_bfloat16 *gz, const __nv_bfloat16 *x,
                                                    float *gw, int L, int C, int k, int dil)
{
    __shared__ float gs[kSimtTX][kSimtTC + 1];
    __shared__ float xs[kSimtMaxSpan][kSimtCI + 1];
    const int tid = threadIdx.x, x0 = blockIdx.x * kSimtTX, b = blockIdx.z;
    const int ntc = C / kSimtTC;
    const int co0 = (blockIdx.y % ntc) * kSimtTC, ci0 = (blockIdx.y / ntc) * kSimtCI;
    const int half = k / 2, span = kSimtTX + (k - 1) * dil;
    for (int e = tid; e < kSimtTX * kSimtTC; e += 256) {
        const int r = e / kSimtTC, o = e % kSimtTC, l = x0 + r;
        gs[r][o] = l < L ? __bfloat162float(gz[((int64_t)b * L + l) * C + co0 + o]) : 0.f;
    }
    for (int e = tid; e < span * kSimtCI; e += 256) {
        const int r = e / kSimtCI, c = e % kSimtCI, l = x0 - half * dil + r;
        xs[r][c] = (l >= 0 && l < L) ? __bfloat162float(x[((int64_t)b * L + l) * C + ci0 + c]) : 0.f;
    }
    __syncthreads();
    for (int pair = tid; pair < kSimtTC * kSimtCI; pair += 256) {
        const int o = pair / kSimtCI, c = pair % kSimtCI;
        for (int t = 0; t < k; ++t) {
            float sum = 0.f;
            for (int r = 0; r < kSimtTX; ++r) sum = fmaf(gs[r][o], xs[r + t * dil][c], sum);
            atomicAdd(&gw[((int64_t)t * C + co0 + o) * C + ci0 + c], sum);
        }
    }
}

// ------------------------------------------------------------ small kernels
int grid_for(int64_t n, int threads = 256)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 152 * 16));
}

// x0[p][c] = bf16(sum_j feat[p][j] Wl[c][j] + bl[c]).  A block of C threads
// takes a range of positions: it first copies their feature rows to shared
// memory with coalesced 16-byte loads, then thread t forms channels 2(t mod
// C/2) and 2(t mod C/2) + 1 (their weight rows in registers) of every other
// position from broadcast reads, so a warp stores 64 consecutive channels of
// a position (128 bytes) per instruction.
template <int F>
__global__ void k_lift(const float *feat, const float *Wl, const float *bl, __nv_bfloat16 *x0,
                       int64_t P, int C, int64_t per_block)
{
    extern __shared__ float4 fsh[];  // [per_block][F / 4]
    const int half = C / 2;
    const int cp = threadIdx.x % half, par = threadIdx.x / half, c = 2 * cp;
    float w0[F], w1[F];
#pragma unroll
    for (int j = 0; j < F / 4; ++j) {
        const float4 q0 = __ldg(reinterpret_cast<const float4 *>(Wl + c * F) + j);
        const float4 q1 = __ldg(reinterpret_cast<const float4 *>(Wl + (c + 1) * F) + j);
        w0[4 * j] = q0.x, w0[4 * j + 1] = q0.y, w0[4 * j + 2] = q0.z, w0[4 * j + 3] = q0.w;
        w1[4 * j] = q1.x, w1[4 * j + 1] = q1.y, w1[4 * j + 2] = q1.z, w1[4 * j + 3] = q1.w;
    }
    const float bias0 = bl[c], bias1 = bl[c + 1];
    const int64_t p0 = blockIdx.x * per_block, p1 = std::min(P, p0 + per_block);
    const int n4 = (int)(p1 - p0) * (F / 4);
    const float4 *src = reinterpret_cast<const float4 *>(feat + p0 * F);
    for (int e = threadIdx.x; e < n4; e += blockDim.x) fsh[e] = __ldg(src + e);
    __syncthreads();
    for (int64_t p = p0 + par; p < p1; p += 2) {
        const float4 *f = fsh + (p - p0) * (F / 4);
        float acc0 = bias0, acc1 = bias1;
#pragma unroll
        for (int j = 0; j < F / 4; ++j) {
            const float4 v = f[j];
            acc0 = fmaf(v.x, w0[4 * j], acc0);
            acc0 = fmaf(v.y, w0[4 * j + 1], acc0);
            acc0 = fmaf(v.z, w0[4 * j + 2], acc0);
            acc0 = fmaf(v.w, w0[4 * j + 3], acc0);
            acc1 = fmaf(v.x, w1[4 * j], acc1);
            acc1 = fmaf(v.y, w1[4 * j + 1], acc1);
            acc1 = fmaf(v.z, w1[4 * j + 2], acc1);
            acc1 = fmaf(v.w, w1[4 * j + 3], acc1);
        }
        *reinterpret_cast<__nv_bfloat162 *>(x0 + p * C + c) = __floats2bfloat162_rn(acc0, acc1);
    }
}

// out[p][o] = sum_c x[p][c] Wp[o][c] + bp[o]: one thread per position reads
// its row of C bf16 values as 16-byte vectors; the FO x C weights sit in
// shared memory and are read as warp-wide broadcasts.
template <int FO>
__global__ void k_head(const __nv_bfloat16 *x, const float *Wp, const float *bp, float *out,
                       int64_t P, int C)
{
    extern __shared__ float wsh[];  // [FO][C]
    for (int i = threadIdx.x; i < FO * C; i += blockDim.x) wsh[i] = Wp[i];
    __syncthreads();
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= P) return;
    float acc[FO];
#pragma unroll
    for (int o = 0; o < FO; ++o) acc[o] = __ldg(bp + o);
    const uint4 *row = reinterpret_cast<const uint4 *>(x + p * C);
    for (int c8 = 0; c8 < C / 8; ++c8) {
        float xv[8];
        unpack8(__ldg(row + c8), xv);
#pragma unroll
        for (int o = 0; o < FO; ++o) {
            const float4 w0 = *reinterpret_cast<const float4 *>(wsh + o * C + 8 * c8);
            const float4 w1 = *reinterpret_cast<const float4 *>(wsh + o * C + 8 * c8 + 4);
            acc[o] = fmaf(xv[0], w0.x, acc[o]);
            acc[o] = fmaf(xv[1], w0.y, acc[o]);
            acc[o] = fmaf(xv[2], w0.z, acc[o]);
            acc[o] = fmaf(xv[3], w0.w, acc[o]);
            acc[o] = fmaf(xv[4], w1.x, acc[o]);
            acc[o] = fmaf(xv[5], w1.y, acc[o]);
            acc[o] = fmaf(xv[6], w1.z, acc[o]);
            acc[o] = fmaf(xv[7], w1.w, acc[o]);
        }
    }
#pragma unroll
    for (int o = 0; o < FO; ++o) out[p * FO + o] = acc[o];
}

// Head backward: gx = gout Wp; gz = bf16(gx gelu'(z)); gWp += gout^T x; gbp += sum gout.
// One warp per position, lane holding channels lane + 32 j (NJ = C / 32),
// FO outputs: both compile-time so that the partial sums stay in registers
// (the head weights are read through L1).
template <int NJ, int FO>
__global__ void k_head_bwd(const float *gout, const __nv_bfloat16 *x, const float *Wp,
                           const __nv_bfloat16 *z, float *gx, __nv_bfloat16 *gz, float *gWp,
                           float *gbp, int64_t P)
{
    constexpr int C = 32 * NJ;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    float accW[FO][NJ], accB[FO];
#pragma unroll
    for (int o = 0; o < FO; ++o) {
        accB[o] = 0.f;
#pragma unroll
        for (int j = 0; j < NJ; ++j) accW[o][j] = 0.f;
    }
    for (int64_t p = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); p < P; p += warps) {
        float go[FO];
#pragma unroll
        for (int o = 0; o < FO; ++o) {
            go[o] = __ldg(gout + p * FO + o);
            accB[o] += go[o];
        }
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            const int64_t c = p * C + lane + 32 * j;
            const float xv = __bfloat162float(x[c]);
            float g = 0.f;
#pragma unroll
            for (int o = 0; o < FO; ++o) {
                g = fmaf(go[o], __ldg(Wp + o * C + lane + 32 * j), g);
                accW[o][j] = fmaf(go[o], xv, accW[o][j]);
            }
            gx[c] = g;
            gz[c] = __float2bfloat16_rn(g * gelu_grad(__bfloat162float(z[c])));
        }
    }
#pragma unroll
    for (int o = 0; o < FO; ++o) {
#pragma unroll
        for (int j = 0; j < NJ; ++j) atomicAdd(&gWp[o * C + lane + 32 * j], accW[o][j]);
        if (lane == 0) atomicAdd(&gbp[o], accB[o]);
    }
}

// Lift backward: gWl[c][j] += sum_p gx0[p][c] feat[p][j]; gbl[c] += sum_p gx0[p][c].
// Threads over channels, blocks over position ranges, F features compile-time.
template <int F>
__global__ void k_lift_bwd(const float *gx0, const float *feat, float *gWl, float *gbl, int64_t P,
                           int C, int64_t per_block)
{
    const int c = threadIdx.x;  // blockDim.x == C
    float acc[F];
#pragma unroll
    for (int j = 0; j < F; ++j) acc[j] = 0.f;
    float accb = 0.f;
    const int64_t p0 = blockIdx.x * per_block, p1 = std::min(P, p0 + per_block);
    for (int64_t p = p0; p < p1; ++p) {
        const float g = gx0[p * C + c];
        accb += g;
#pragma unroll
        for (int j = 0; j < F; ++j) acc[j] = fmaf(g, __ldg(feat + p * F + j), acc[j]);
    }
#pragma unroll
    for (int j = 0; j < F; ++j) atomicAdd(&gWl[c * F + j], acc[j]);
    atomicAdd(&gbl[c], accb);
}

// gb[c] += sum_p gz[p][c] (bf16 input), threads over channels
__global__ void k_colsum(const __nv_bfloat16 *gz, float *gb, int64_t P, int C, int64_t per_block)
{
    const int64_t p0 = blockIdx.x * per_block, p1 = std::min(P, p0 + per_block);
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        float s = 0.f;
        for (int64_t p = p0; p < p1; ++p) s += __bfloat162float(gz[p * C + c]);
        atomicAdd(&gb[c], s);
    }
}

// bf16 copies of the fp32 conv weights: W[t][co][ci] and WT[t][ci][co] = W[k-1-t][co][ci]
__global__ void k_cast_weights(const float *w, __nv_bfloat16 *wb, __nv_bfloat16 *wt, int C, int k,
                               int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t per_layer = (int64_t)k * C * C;
        const int64_t layer = i / per_layer, r = i % per_layer;
        const int t = (int)(r / ((int64_t)C * C)), co = (int)((r / C) % C), ci = (int)(r % C);
        const __nv_bfloat16 v = __float2bfloat16_rn(w[i]);
        wb[i] = v;
        if (wt) wt[layer * per_layer + ((int64_t)(k - 1 - t) * C + ci) * C + co] = v;
    }
}

__global__ void k_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1,
                       float b2, float eps, float c1, float c2, float wd)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i] + wd * p[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

// Adam's per-step constants from a device step counter, so that a captured
// training step replays with the right learning rate and bias corrections:
// t = ++*step; hyper = (lr_table[min(t, len) - 1], 1 / (1 - b1^t), 1 / (1 - b2^t)).
__global__ void k_adam_prep(int64_t *step, const float *lr_table, int64_t len, float b1, float b2,
                            float *hyper)
{
    const int64_t t = ++*step;
    hyper[0] = lr_table[(t < len ? t : len) - 1];
    hyper[1] = (float)(1.0 / (1.0 - pow((double)b1, (double)t)));
    hyper[2] = (float)(1.0 / (1.0 - pow((double)b2, (double)t)));
}

__global__ void k_adam_dev(float *p, const float *g, float *m, float *v, int64_t n,
                           const float *hyper, float b1, float b2, float eps, float wd)
{
    const float lr = hyper[0], c1 = hyper[1], c2 = hyper[2];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i] + wd * p[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

// SplitMix64 (Steele, Lea and Flood, 2014): a counter-based generator, here
// keyed by (seed, step, i).
__device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// Minibatch of training pairs drawn on the device: pair i of the step
// *step takes tube good[h mod ngood] and window j = (h >> 32) mod windows,
// h = splitmix64(seed ^ splitmix64(step * batch + i)); rows index the
// trajectory fields stored window-major ([windows + 1][tubes][L]).
__global__ void k_sample_pairs(const int *good, int ngood, int windows, int tubes,
                               const float *gamma_tubes, uint64_t seed, const int64_t *step,
                               int batch, int64_t *rows_src, int64_t *rows_dst, float *gamma_out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= batch) return;
    const uint64_t h = splitmix64(seed ^ splitmix64((uint64_t)(*step) * (uint64_t)batch + i));
    const int tube = good[(int)((h & 0xFFFFFFFFull) % (uint64_t)ngood)];
    const int j = (int)((h >> 32) % (uint64_t)windows);
    rows_src[i] = (int64_t)j * tubes + tube;
    rows_dst[i] = (int64_t)(j + 1) * tubes + tube;
    gamma_out[i] = gamma_tubes[tube];
}

// loss partial sums (double) and gout = 2 (out - target) / n
__global__ void k_mse(const float *out, const float *target, float *gout, double *loss, int64_t n)
{
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float d = out[i] - target[i];
        acc += (double)d * d;
        if (gout) gout[i] = 2.0f * d / (float)n;
    }
    __shared__ double red[32];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        atomicAdd(loss, s / (double)n);
    }
}

struct Scale4 { float s[4]; };
struct Scale3 { float s[3]; };

// feat[i] = ((rho-1)/s0, u/s1, (T-1)/s2, (gamma_b-1.4)/s3)
__global__ void k_features(const float *rho, const float *u, const float *T, const float *gamma,
                           float *feat, int64_t n, int L, Scale4 sc)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float4 f = make_float4((rho[i] - 1.0f) / sc.s[0], u[i] / sc.s[1], (T[i] - 1.0f) / sc.s[2],
                                     (gamma[i / L] - 1.4f) / sc.s[3]);
        reinterpret_cast<float4 *>(feat)[i] = f;
    }
}

// target[i] = ((rho2-rho)/s0, (u2-u)/s1, (T2-T)/s2)
__global__ void k_targets(const float *rho, const float *u, const float *T, const float *rho2,
                          const float *u2, const float *T2, float *target, int64_t n, Scale3 sc)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        target[3 * i + 0] = (rho2[i] - rho[i]) / sc.s[0];
        target[3 * i + 1] = (u2[i] - u[i]) / sc.s[1];
        target[3 * i + 2] = (T2[i] - T[i]) / sc.s[2];
    }
}

// (rho, u, T)_out = (rho, u, T) + out * scale
__global__ void k_apply(const float *rho, const float *u, const float *T, const float *out,
                        float *rho2, float *u2, float *T2, int64_t n, Scale3 sc)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        rho2[i] = rho[i] + out[3 * i + 0] * sc.s[0];
        u2[i] = u[i] + out[3 * i + 1] * sc.s[1];
        T2[i] = T[i] + out[3 * i + 2] * sc.s[2];
    }
}

// One block per tube: conservation residual between two states (mass,
// momentum scaled by mass, total energy with (1+n)/2 T) and, when a
// reference is given, the L1 error (max over rho, u relative to the sound
// speed, T).  Window [w0, w0 + W) of each tube of length L.  With `starts`,
// also the spot-check window of `span` nodes centred on the node where rho
// changes most: starts[b] = clamp(argmax - span/2, 0, L - span) and
// starts[B + b] = starts[b] + margin.
__global__ void k_tube_checks(const float *rho, const float *u, const float *T, const float *rho2,
                              const float *u2, const float *T2, const float *half_dof,
                              const float *gamma, float *residual, float *l1, int *starts, int L,
                              int w0, int W, int span, int margin)
{
    constexpr int NV = 12;
    __shared__ double red[NV][32];
    __shared__ float best_v[32];
    __shared__ int best_i[32];
    const int b = blockIdx.x;
    const float cv = half_dof ? half_dof[b] : 0.f;  // only read when residual is asked for
    const float g = l1 ? gamma[b] : 0.f;
    // Per node in float, per thread in float (a few tens of terms), across
    // the block in double.  The residual sums accumulate the differences
    // of the two states node by node, so a small change keeps its digits:
    // totals of the first state (mass, momentum, energy), their changes,
    // the L1 differences of rho, u, T and the reference's sound-speed, T
    // and rho sums.
    float s[NV] = {};
    float bv = -1.0f;
    int bi = w0;
    int unphysical = 0;  // a non-positive or non-finite rho or T in the second state
    for (int l = w0 + threadIdx.x; l < w0 + W; l += blockDim.x) {
        const int64_t i = (int64_t)b * L + l;
        const float r1 = rho[i], v1 = u[i], t1 = T[i], r2 = rho2[i], v2 = u2[i], t2 = T2[i];
        if (residual) {
            unphysical |= !(r2 > 0.f) || !(t2 > 0.f) || !(r2 < INFINITY) || !(t2 < INFINITY) ||
                          !isfinite(v2);
            const float j1 = r1 * v1;
            const float e1 = r1 * fmaf(cv, t1, 0.5f * v1 * v1);
            s[0] += r1;
            s[1] += j1;
            s[2] += e1;
            s[3] += r2 - r1;
            s[4] += fmaf(r2, v2, -j1);
            s[5] += fmaf(r2, fmaf(cv, t2, 0.5f * v2 * v2), -e1);
        }
        if (l1) {
            s[6] += fabsf(r1 - r2);
            s[7] += fabsf(v1 - v2);
            s[8] += fabsf(t1 - t2);
            s[9] += sqrtf(g * t2);
            s[10] += fabsf(t2);
            s[11] += fabsf(r2);
        }
        const float d = fabsf(r2 - r1);
        if (!(d <= bv)) {  // also takes a non-finite change
            bv = isfinite(d) ? d : INFINITY;
            bi = l;
        }
    }
    // one block-wide reduction of all the sums
    unphysical = __syncthreads_or(unphysical);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double v = s[q];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) red[q][warp] = v;
    }
    __syncthreads();
    double tot[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        tot[q] = 0.0;
        for (int w = 0; w < nw; ++w) tot[q] += red[q][w];
    }
    const double cs = tot[9], ts = tot[10];
    if (starts) {  // argmax of |rho2 - rho|, smallest index on ties
        for (int off = 16; off > 0; off >>= 1) {
            const float ov = __shfl_down_sync(0xffffffffu, bv, off);
            const int oi = __shfl_down_sync(0xffffffffu, bi, off);
            if (ov > bv || (ov == bv && oi < bi)) bv = ov, bi = oi;
        }
        if ((threadIdx.x & 31) == 0) best_v[threadIdx.x >> 5] = bv, best_i[threadIdx.x >> 5] = bi;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
                if (best_v[w] > bv || (best_v[w] == bv && best_i[w] < bi)) bv = best_v[w], bi = best_i[w];
            const int st = min(max(bi - span / 2, 0), L - span);
            starts[b] = st;
            starts[gridDim.x + b] = st + margin;
        }
    }
    if (threadIdx.x == 0) {
        if (residual) {
            const double m = fabs(tot[3]) / tot[0];
            const double j = fabs(tot[4]) / tot[0];
            const double e = fabs(tot[5]) / tot[2];
            residual[b] = unphysical ? INFINITY : (float)fmax(m, fmax(j, e));
        }
        if (l1) {
            const double er = tot[6] / tot[11];
            const double eu = tot[7] / cs;
            const double et = tot[8] / ts;
            l1[b] = (float)fmax(er, fmax(eu, et));
        }
    }
}

// dst_f[i][w] = src_f[rows[i] * row_len + off[i] + w] for the three fields
// (scatter: the reverse assignment).  One block row per (i, chunk of w).
template <bool SCATTER>
__global__ void k_rows(const float *a, const float *b, const float *c, float *da, float *db,
                       float *dc, const int64_t *rows, const int *off, int count, int64_t row_len,
                       int W)
{
    const int64_t n = (int64_t)count * W;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / W), w = (int)(e % W);
        const int64_t g = rows[i] * row_len + (off ? off[i] : 0) + w;
        if (SCATTER) {
            da[g] = a[e];
            db[g] = b[e];
            dc[g] = c[e];
        } else {
            da[e] = a[g];
            db[e] = b[g];
            dc[e] = c[g];
        }
    }
}

// ------------------------------------------------------------ host helpers
PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// [B][L][C] bf16, box (64 channels, rows positions, 1 tube), 128-byte swizzle
bool map_act(CUtensorMap *m, const void *ptr, int B, int L, int C, int rows)
{
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)C, (cuuint64_t)L, (cuuint64_t)B};
    const cuuint64_t strides[2] = {(cuuint64_t)C * 2, (cuuint64_t)L * C * 2};
    const cuuint32_t box[3] = {(cuuint32_t)kChunk, (cuuint32_t)rows, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(ptr), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// [k*C][C] bf16 weights, box (64 input channels, 128 output rows)
bool map_w(CUtensorMap *m, const void *ptr, int C, int k)
{
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)C, (cuuint64_t)k * C};
    const cuuint64_t strides[1] = {(cuuint64_t)C * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kChunk, (cuuint32_t)kTile};
    const cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

int set_smem_attrs()
{
    // once per device: the dynamic shared-memory limit of the three kernels
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return LBM_ECUDA;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return LBM_OK;
    if (cudaFuncSetAttribute(k_conv_tc<kEpiForward>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kSmemBytes) != cudaSuccess ||
        cudaFuncSetAttribute(k_conv_tc<kEpiInputGrad>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kSmemBytes) != cudaSuccess ||
        cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_conv_tcp<kEpiForward>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kPSmemBytes) != cudaSuccess ||
        cudaFuncSetAttribute(k_conv_tcp<kEpiInputGrad>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kPSmemBytes) != cudaSuccess ||
        cudaFuncSetAttribute(k_conv_tcn<kEpiForward>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kNSmemMax) != cudaSuccess ||
        cudaFuncSetAttribute(k_conv_tcn<kEpiInputGrad>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kNSmemMax) != cudaSuccess)
        return LBM_ECUDA;
    done[dev] = true;
    return LBM_OK;
}

int launched(cudaError_t e) { return e == cudaSuccess ? LBM_OK : LBM_ECUDA; }

bool conv_shape_ok(int B, int L, int C, int k, int dil, int impl)
{
    if (B < 1 || B > 65535 || L < 1 || C < 128 || C % 128 != 0 || k < 1 || k % 2 == 0 || dil < 1)
        return false;
    if ((int64_t)(k / 2) * dil >= (1 << 20) || (int64_t)B * L * C >= (1ll << 40)) return false;
    if (impl == 1) return k <= kSimtMaxK && (k - 1) * dil <= kSimtMaxSpan - kSimtTX;
    if (impl == 3) return (int64_t)(k - 1) * dil <= kMaxHalo && (int64_t)k * C <= (1 << 20);
    return (impl == 0 || impl == 2) && (int64_t)k * C <= (1 << 20);
}

// SM count of the current device, looked up once per device (so that calls
// made while a stream is being captured into a graph query nothing)
int sm_count()
{
    static std::mutex mu;
    static int count[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    std::lock_guard<std::mutex> lock(mu);
    if (count[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
            return 0;
        count[dev] = n;
    }
    return count[dev];
}

int conv_common(int epi, const void *in, const void *w, const ConvArgs &a, int impl, void *stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    if (impl == 1) {
        const dim3 grid((a.L + kSimtTX - 1) / kSimtTX, a.C / kSimtTC, a.B);
        if (epi == kEpiForward)
            k_conv_simt<kEpiForward><<<grid, 256, 0, s>>>((const __nv_bfloat16 *)in,
                                                          (const __nv_bfloat16 *)w, a);
        else
            k_conv_simt<kEpiInputGrad><<<grid, 256, 0, s>>>((const __nv_bfloat16 *)in,
                                                            (const __nv_bfloat16 *)w, a);
        return launched(cudaGetLastError());
    }
    if (!aligned16(in) || !aligned16(w)) return LBM_EINVAL;
    int rc = set_smem_attrs();
    if (rc != LBM_OK) return rc;
    CUtensorMap ma, mw;
    if (impl == 3) {  // persistent, channels x 256 positions per tile
        const int rows = window_rows(a.k, a.dil);
        if (!map_act(&ma, in, a.B, a.L, a.C, rows / 2) || !map_w(&mw, w, a.C, a.k)) return LBM_ECUDA;
        const int tiles_l = (a.L + kNPos - 1) / kNPos, tiles_m = a.C / kTile;
        const int64_t total = (int64_t)tiles_l * tiles_m * a.B;
        const int sms = sm_count();
        if (sms < 1 || total >= (1ll << 31)) return LBM_ECUDA;
        const int grid = (int)std::min<int64_t>(total, sms);
        const int smem = tcn_smem_bytes(rows);
        if (epi == kEpiForward)
            k_conv_tcn<kEpiForward><<<grid, kPThreads, smem, s>>>(ma, mw, a, tiles_l, tiles_m,
                                                                  (int)total, rows);
        else
            k_conv_tcn<kEpiInputGrad><<<grid, kPThreads, smem, s>>>(ma, mw, a, tiles_l, tiles_m,
                                                                    (int)total, rows);
        return launched(cudaGetLastError());
    }
    if (!map_act(&ma, in, a.B, a.L, a.C, kTile) || !map_w(&mw, w, a.C, a.k)) return LBM_ECUDA;
    const int tiles_l = (a.L + kTile - 1) / kTile, tiles_n = a.C / kTile;
    if (impl == 2) {  // one output tile per block
        const dim3 grid(tiles_l, tiles_n, a.B);
        if (epi == kEpiForward)
            k_conv_tc<kEpiForward><<<grid, 128, kSmemBytes, s>>>(ma, mw, a);
        else
            k_conv_tc<kEpiInputGrad><<<grid, 128, kSmemBytes, s>>>(ma, mw, a);
        return launched(cudaGetLastError());
    }
    const int64_t total = (int64_t)tiles_l * tiles_n * a.B;
    const int sms = sm_count();
    if (sms < 1 || total >= (1ll << 31)) return LBM_ECUDA;
    const int grid = (int)std::min<int64_t>(total, sms);
    if (epi == kEpiForward)
        k_conv_tcp<kEpiForward><<<grid, kPThreads, kPSmemBytes, s>>>(ma, mw, a, tiles_l, tiles_n,
                                                                      (int)total);
    else
        k_conv_tcp<kEpiInputGrad><<<grid, kPThreads, kPSmemBytes, s>>>(ma, mw, a, tiles_l, tiles_n,
                                                                        (int)total);
    return launched(cudaGetLastError());
}

}  // namespace

extern "C" {

int lbm_nn_conv_forward(const void *x, const void *w, const float *bias, void *y, void *z, int B,
                        int L, int C, int k, int dil, int impl, int *status, void *stream)
{
    if (!x || !w || !bias || !y || !conv_shape_ok(B, L, C, k, dil, impl) || x == y) return LBM_EINVAL;
    if (!aligned16(y) || (z && !aligned16(z))) return LBM_EINVAL;
    ConvArgs a{};
    a.B = B, a.L = L, a.C = C, a.k = k, a.dil = dil;
    a.x = (const __nv_bfloat16 *)x;
    a.bias = bias;
    a.y = (__nv_bfloat16 *)y;
    a.z = (__nv_bfloat16 *)z;
    a.status = status;
    return conv_common(kEpiForward, x, w, a, impl, stream);
}

int lbm_nn_conv_backward_data(const void *gz, const void *wt, float *gx, const void *zprev,
                              void *gzprev, int B, int L, int C, int k, int dil, int impl,
                              int *status, void *stream)
{
    if (!gz || !wt || !gx || !conv_shape_ok(B, L, C, k, dil, impl)) return LBM_EINVAL;
    if ((zprev == nullptr) != (gzprev == nullptr) || gzprev == gz) return LBM_EINVAL;
    if (!aligned16(gx) || (zprev && (!aligned16(zprev) || !aligned16(gzprev)))) return LBM_EINVAL;
    ConvArgs a{};
    a.B = B, a.L = L, a.C = C, a.k = k, a.dil = dil;
    a.gx = gx;
    a.zprev = (const __nv_bfloat16 *)zprev;
    a.gzprev = (__nv_bfloat16 *)gzprev;
    a.status = status;
    return conv_common(kEpiInputGrad, gz, wt, a, impl, stream);
}

int lbm_nn_conv_backward_weight(const void *gz, const void *x, float *gw, int B, int L, int C, int k,
                                int dil, int impl, int *status, void *stream)
{
    if (!gz || !x || !gw || !conv_shape_ok(B, L, C, k, dil, impl)) return LBM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (impl == 1) {
        const dim3 grid((L + kSimtTX - 1) / kSimtTX, (C / kSimtTC) * (C / kSimtCI), B);
        k_wgrad_simt<<<grid, 256, 0, s>>>((const __nv_bfloat16 *)gz, (const __nv_bfloat16 *)x, gw,
                                          L, C, k, dil);
        return launched(cudaGetLastError());
    }
    if (!aligned16(gz) || !aligned16(x) || !aligned16(gw)) return LBM_EINVAL;
    int rc = set_smem_attrs();
    if (rc != LBM_OK) return rc;
    CUtensorMap mg, mx;
    if (!map_act(&mg, gz, B, L, C, kWgRows) || !map_act(&mx, x, B, L, C, kWgRows)) return LBM_ECUDA;
    const int tiles = (C / kTile) * (C / kTile) * k;
    const int64_t total = (int64_t)B * ((L + kWgRows - 1) / kWgRows);
    // about two resident blocks per SM in one wave
    const int64_t want = std::max<int64_t>(1, (2 * 152 + tiles - 1) / tiles);
    const int per_block = (int)std::max<int64_t>(1, (total + want - 1) / want);
    const int chunks = (int)((total + per_block - 1) / per_block);
    k_wgrad_tc<<<dim3(chunks, tiles), 128, kSmemBytes, s>>>(mg, mx, gw, B, L, C, k, dil, per_block,
                                                            status);
    return launched(cudaGetLastError());
}

int lbm_nn_cast_weights(const float *w, void *w_bf16, void *wt_bf16, int layers, int C, int k,
                        void *stream)
{
    if (!w || !w_bf16 || layers < 1 || C < 1 || k < 1) return LBM_EINVAL;
    const int64_t n = (int64_t)layers * k * C * C;
    k_cast_weights<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(w, (__nv_bfloat16 *)w_bf16,
                                                                  (__nv_bfloat16 *)wt_bf16, C, k, n);
    return launched(cudaGetLastError());
}

int lbm_nn_lift(const float *feat, const float *Wl, const float *bl, void *x0, int64_t P, int F,
                int C, void *stream)
{
    if (!feat || !Wl || !bl || !x0 || P < 1 || C < 32 || C > 1024 || C % 32 ||
        (F != 4 && F != 8 && F != 16 && F != 32) || !aligned16(feat) || !aligned16(Wl))
        return LBM_EINVAL;
    const int64_t per_block = 256;  // feature rows staged per block: 4 KB to 32 KB
    const int64_t nblocks = (P + per_block - 1) / per_block;
    if (nblocks > 0x7fffffff) return LBM_EINVAL;
    const int blocks = (int)nblocks;
    const size_t sh = (size_t)per_block * F * sizeof(float);
    cudaStream_t s = (cudaStream_t)stream;
    auto out = (__nv_bfloat16 *)x0;
    switch (F) {
    case 4: k_lift<4><<<blocks, C, sh, s>>>(feat, Wl, bl, out, P, C, per_block); break;
    case 8: k_lift<8><<<blocks, C, sh, s>>>(feat, Wl, bl, out, P, C, per_block); break;
    case 16: k_lift<16><<<blocks, C, sh, s>>>(feat, Wl, bl, out, P, C, per_block); break;
    default: k_lift<32><<<blocks, C, sh, s>>>(feat, Wl, bl, out, P, C, per_block); break;
    }
    return launched(cudaGetLastError());
}

int lbm_nn_lift_backward(const float *gx0, const float *feat, float *gWl, float *gbl, int64_t P,
                         int F, int C, void *stream)
{
    if (!gx0 || !feat || !gWl || !gbl || P < 1 || C < 32 || C > 1024 || C % 32 ||
        (F != 4 && F != 8 && F != 16 && F != 32))
        return LBM_EINVAL;
    const int64_t per_block = std::max<int64_t>(64, (P + 1215) / 1216);
    const int blocks = (int)((P + per_block - 1) / per_block);
    cudaStream_t s = (cudaStream_t)stream;
    switch (F) {
    case 4: k_lift_bwd<4><<<blocks, C, 0, s>>>(gx0, feat, gWl, gbl, P, C, per_block); break;
    case 8: k_lift_bwd<8><<<blocks, C, 0, s>>>(gx0, feat, gWl, gbl, P, C, per_block); break;
    case 16: k_lift_bwd<16><<<blocks, C, 0, s>>>(gx0, feat, gWl, gbl, P, C, per_block); break;
    default: k_lift_bwd<32><<<blocks, C, 0, s>>>(gx0, feat, gWl, gbl, P, C, per_block); break;
    }
    return launched(cudaGetLastError());
}

int lbm_nn_head(const void *x, const float *Wp, const float *bp, float *out, int64_t P, int C, int Fo,
                void *stream)
{
    if (!x || !Wp || !bp || !out || P < 1 || C < 8 || C > 1024 || C % 8 || !aligned16(x) ||
        !aligned16(Wp) || (Fo != 3 && Fo != 6 && Fo != 12 && Fo != 24))
        return LBM_EINVAL;
    const int64_t nblocks = (P + 127) / 128;
    if (nblocks > 0x7fffffff) return LBM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    auto xb = (const __nv_bfloat16 *)x;
    const size_t sh = sizeof(float) * Fo * C;
    if (Fo == 3) k_head<3><<<(int)nblocks, 128, sh, s>>>(xb, Wp, bp, out, P, C);
    else if (Fo == 6) k_head<6><<<(int)nblocks, 128, sh, s>>>(xb, Wp, bp, out, P, C);
    else if (Fo == 12) k_head<12><<<(int)nblocks, 128, sh, s>>>(xb, Wp, bp, out, P, C);
    else k_head<24><<<(int)nblocks, 128, sh, s>>>(xb, Wp, bp, out, P, C);
    return launched(cudaGetLastError());
}

int lbm_nn_head_backward(const float *gout, const void *x, const float *Wp, const void *z, float *gx,
                         void *gz, float *gWp, float *gbp, int64_t P, int C, int Fo, void *stream)
{
    if (!gout || !x || !Wp || !z || !gx || !gz || !gWp || !gbp || P < 1 ||
        (C != 128 && C != 256) || (Fo != 3 && Fo != 6 && Fo != 12 && Fo != 24))
        return LBM_EINVAL;
    const int grid = (int)std::min<int64_t>(grid_for(P * 32), 152 * 4);
    cudaStream_t s = (cudaStream_t)stream;
    auto xb = (const __nv_bfloat16 *)x;
    auto zb = (const __nv_bfloat16 *)z;
    auto gzb = (__nv_bfloat16 *)gz;
#define LBM_HEAD_BWD(NJ, FO) \
    k_head_bwd<NJ, FO><<<grid, 256, 0, s>>>(gout, xb, Wp, zb, gx, gzb, gWp, gbp, P)
    if (C == 128) {
        if (Fo == 3) LBM_HEAD_BWD(4, 3);
        else if (Fo == 6) LBM_HEAD_BWD(4, 6);
        else if (Fo == 12) LBM_HEAD_BWD(4, 12);
        else LBM_HEAD_BWD(4, 24);
    } else {
        if (Fo == 3) LBM_HEAD_BWD(8, 3);
        else if (Fo == 6) LBM_HEAD_BWD(8, 6);
        else if (Fo == 12) LBM_HEAD_BWD(8, 12);
        else LBM_HEAD_BWD(8, 24);
    }
#undef LBM_HEAD_BWD
    return launched(cudaGetLastError());
}

int lbm_nn_bias_grad(const void *gz, float *gb, int64_t P, int C, void *stream)
{
    if (!gz || !gb || P < 1 || C < 1) return LBM_EINVAL;
    const int64_t per_block = std::max<int64_t>(64, (P + 1215) / 1216);
    const int blocks = (int)((P + per_block - 1) / per_block);
    k_colsum<<<blocks, std::min(C, 256), 0, (cudaStream_t)stream>>>((const __nv_bfloat16 *)gz, gb, P,
                                                                    C, per_block);
    return launched(cudaGetLastError());
}

int lbm_nn_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                float eps, int t, float weight_decay, void *stream)
{
    if (!p || !g || !m || !v || n < 1 || t < 1) return LBM_EINVAL;
    const float c1 = (float)(1.0 / (1.0 - std::pow((double)b1, t)));
    const float c2 = (float)(1.0 / (1.0 - std::pow((double)b2, t)));
    k_adam<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2,
                                                          weight_decay);
    return launched(cudaGetLastError());
}

int lbm_nn_adam_scheduled(float *p, const float *g, float *m, float *v, int64_t n,
                          const float *lr_table, int64_t table_len, int64_t *step, float *hyper,
                          float b1, float b2, float eps, float weight_decay, void *stream)
{
    if (!p || !g || !m || !v || !lr_table || !step || !hyper || n < 1 || table_len < 1)
        return LBM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    k_adam_prep<<<1, 1, 0, s>>>(step, lr_table, table_len, b1, b2, hyper);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return LBM_ECUDA;
    k_adam_dev<<<grid_for(n), 256, 0, s>>>(p, g, m, v, n, hyper, b1, b2, eps, weight_decay);
    return launched(cudaGetLastError());
}

int lbm_nn_sample_pairs(const int *good, int ngood, int windows, int tubes,
                        const float *gamma_tubes, uint64_t seed, const int64_t *step, int batch,
                        int64_t *rows_src, int64_t *rows_dst, float *gamma_out, void *stream)
{
    if (!good || ngood < 1 || windows < 1 || tubes < 1 || !gamma_tubes || !step || batch < 1 ||
        !rows_src || !rows_dst || !gamma_out)
        return LBM_EINVAL;
    k_sample_pairs<<<(batch + 127) / 128, 128, 0, (cudaStream_t)stream>>>(
        good, ngood, windows, tubes, gamma_tubes, seed, step, batch, rows_src, rows_dst, gamma_out);
    return launched(cudaGetLastError());
}

int lbm_nn_mse(const float *out, const float *target, float *gout, double *loss, int64_t n,
               void *stream)
{
    if (!out || !target || !loss || n < 1) return LBM_EINVAL;
    k_mse<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(out, target, gout, loss, n);
    return launched(cudaGetLastError());
}

int lbm_nn_features(const float *rho, const float *u, const float *T, const float *gamma, float *feat,
                    int B, int L, const float *in_scale, void *stream)
{
    if (!rho || !u || !T || !gamma || !feat || !in_scale || B < 1 || L < 1 || !aligned16(feat))
        return LBM_EINVAL;
    Scale4 sc;
    for (int i = 0; i < 4; ++i) sc.s[i] = in_scale[i];
    const int64_t n = (int64_t)B * L;
    k_features<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(rho, u, T, gamma, feat, n, L, sc);
    return launched(cudaGetLastError());
}

int lbm_nn_targets(const float *rho, const float *u, const float *T, const float *rho2,
                   const float *u2, const float *T2, float *target, int64_t n,
                   const float *out_scale, void *stream)
{
    if (!rho || !u || !T || !rho2 || !u2 || !T2 || !target || !out_scale || n < 1) return LBM_EINVAL;
    Scale3 sc;
    for (int i = 0; i < 3; ++i) sc.s[i] = out_scale[i];
    k_targets<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(rho, u, T, rho2, u2, T2, target, n, sc);
    return launched(cudaGetLastError());
}

int lbm_nn_apply(const float *rho, const float *u, const float *T, const float *out, float *rho2,
                 float *u2, float *T2, int64_t n, const float *out_scale, void *stream)
{
    if (!rho || !u || !T || !out || !rho2 || !u2 || !T2 || !out_scale || n < 1) return LBM_EINVAL;
    Scale3 sc;
    for (int i = 0; i < 3; ++i) sc.s[i] = out_scale[i];
    k_apply<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(rho, u, T, out, rho2, u2, T2, n, sc);
    return launched(cudaGetLastError());
}

int lbm_nn_tube_checks(const float *rho, const float *u, const float *T, const float *rho2,
                       const float *u2, const float *T2, const float *half_dof, const float *gamma,
                       float *residual, float *l1, int *starts, int span, int margin, int B, int L,
                       int w0, int W, void *stream)
{
    if (!rho || !u || !T || !rho2 || !u2 || !T2 || B < 1 || L < 1 || w0 < 0 || W < 1 ||
        w0 + W > L || (!residual && !l1 && !starts) || (residual && !half_dof) || (l1 && !gamma))
        return LBM_EINVAL;
    if (starts && (span < 1 || span > L || margin < 0 || 2 * margin > span)) return LBM_EINVAL;
    k_tube_checks<<<B, 256, 0, (cudaStream_t)stream>>>(rho, u, T, rho2, u2, T2, half_dof, gamma,
                                                       residual, l1, starts, L, w0, W, span, margin);
    return launched(cudaGetLastError());
}


int lbm_nn_wait_selftest(long long budget_cycles, int arrive, int *status, void *stream)
{
    if (!status || budget_cycles < 0 || budget_cycles > (1ll << 34)) return LBM_EINVAL;
    k_wait_selftest<<<1, 32, 0, (cudaStream_t)stream>>>(budget_cycles, arrive, status);
    return launched(cudaGetLastError());
}

int lbm_nn_gather(const float *a, const float *b, const float *c, const int64_t *rows,
                  const int *offsets, int count, int64_t row_len, int W, float *da, float *db,
                  float *dc, void *stream)
{
    if (!a || !b || !c || !rows || !da || !db || !dc || count < 1 || W < 1 || row_len < W)
        return LBM_EINVAL;
    k_rows<false><<<grid_for((int64_t)count * W), 256, 0, (cudaStream_t)stream>>>(
        a, b, c, da, db, dc, rows, offsets, count, row_len, W);
    return launched(cudaGetLastError());
}

int lbm_nn_scatter(const float *a, const float *b, const float *c, const int64_t *rows,
                   const int *offsets, int count, int64_t row_len, int W, float *da, float *db,
                   float *dc, void *stream)
{
    if (!a || !b || !c || !rows || !da || !db || !dc || count < 1 || W < 1 || row_len < W)
        return LBM_EINVAL;
    k_rows<true><<<grid_for((int64_t)count * W), 256, 0, (cudaStream_t)stream>>>(
        a, b, c, da, db, dc, rows, offsets, count, row_len, W);
    return launched(cudaGetLastError());
}

}  // extern "C"
