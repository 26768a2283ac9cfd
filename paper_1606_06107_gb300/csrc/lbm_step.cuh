// Device code of the decoupled Hermite-expansion LBM (arXiv 1606.06107) for
// sm_103a.  Included by one translation unit per lattice, which instantiates
// the kernels for that lattice and defines its launch_<lattice>() entry.
//
// Memory layout in HBM: structure of arrays, population-major.  The state
// buffer holds Q_t translational arrays then Q_r rotational arrays, each of
// S = pitch * Y * Z floats, x fastest, rows padded to a multiple of 32 floats
// (128 bytes) so every row starts on a cache-line boundary.  Element indices
// are 32-bit (the host rejects buffers of 2^31 floats or more), so each load
// address is one 3-input add plus one wide multiply-add.
//
// The step is memory bound: every population is read once and written once
// per step; all moments and equilibria live in registers.  Populations are
// stored as float, as __half / __nv_bfloat16 deviations from rest (Storage
// below), or as deviations from a per-node reference (NodeHalf / NodeBf16,
// with a record per node after the populations; their step kernel is in
// lbm_step_node.cuh); every kernel is instantiated per storage type.  One
// thread owns one node; a block is 128 consecutive x positions of one row.
#pragma once
#include <cstdint>
#include <type_traits>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lbm_internal.h"

namespace lbm {

// Threads per block (x positions of one row).  On the 2048^2 D2Q49 float
// step, with the register cap held at 128 by the resident-block count:
// 128 threads 12,855 Mnode/s, 64 at 8 blocks 12,806, 256 at 2 12,714, 512
// at 1 10,502.
#ifndef LBM_BLOCK_X
#define LBM_BLOCK_X 128
#endif
constexpr int kBlockX = LBM_BLOCK_X;

// Minimum resident blocks per SM requested from the compiler for the step
// kernel, by storage type.  float: 4 caps the D2Q49 kernel at 128 registers
// without spills; measured 4 % faster than letting the compiler choose and
// 4-13 % faster than 3 or 5 on the 2048^2 workload.  half/bfloat16
// deviations in STREAM mode (more instructions per population, half the
// bytes): 5 blocks measured 9 % (f16) and 13 % (bf16) faster than 4 on the
// same workload, 3 slower, 6 no better; FD mode keeps 4 (at 5 its rotational
// variant spills 256 bytes).  LBM_STEP_MIN_BLOCKS overrides all (A/B builds).
template <typename ST, int MODE> struct StepMinBlocks {
#ifdef LBM_STEP_MIN_BLOCKS
    static constexpr int value = LBM_STEP_MIN_BLOCKS;
#else
    static constexpr int value = (std::is_same<ST, float>::value || MODE != 0) ? 4 : 5;
#endif
};
#define LBM_STEP_BOUNDS __launch_bounds__(kBlockX, StepMinBlocks<ST, MODE>::value)

// ---------------------------------------------------------------------------
// Velocity sets.  xi_i = r * e_i; order (ez, ey, ex) ascending.  The sets are
// point symmetric, so in this order population Q-1-i has velocity -e_i and
// the rest velocity sits at the centre index (Q-1)/2; (+-1,0,0) are its
// neighbours.

template <int LAT> struct Lattice;

template <> struct Lattice<1> {  // D1Q7 (Table II)
    static constexpr int D = 1, Q = 7;
    __host__ __device__ static constexpr int ex(int i) { return i - 3; }
    __host__ __device__ static constexpr int ey(int) { return 0; }
    __host__ __device__ static constexpr int ez(int) { return 0; }
};

template <> struct Lattice<3> {  // D2Q49 = D1Q7 x D1Q7
    static constexpr int D = 2, Q = 49;
    __host__ __device__ static constexpr int ex(int i) { return i % 7 - 3; }
    __host__ __device__ static constexpr int ey(int i) { return i / 7 - 3; }
    __host__ __device__ static constexpr int ez(int) { return 0; }
};

// D2Q37 (Table I): the 8 symmetry groups (0,0), (r,0), (r,r), (2r,0),
// (2r,r), (3r,0), (3r,r), (3r,3r) -- the D2Q49 square without the 12
// velocities whose |components| are (2,2), (2,3) or (3,2).
struct D2Q37Table {
    int x[37], y[37];
};
__host__ __device__ constexpr bool d2q37_member(int ex, int ey)
{
    int a = ex < 0 ? -ex : ex, b = ey < 0 ? -ey : ey;
    return !((a == 2 && b == 2) || (a == 2 && b == 3) || (a == 3 && b == 2));
}
__host__ __device__ constexpr D2Q37Table make_d2q37()
{
    D2Q37Table t{};
    int q = 0;
    for (int ey = -3; ey <= 3; ++ey)
        for (int ex = -3; ex <= 3; ++ex)
            if (d2q37_member(ex, ey)) {
                t.x[q] = ex;
                t.y[q] = ey;
                ++q;
            }
    return t;
}
template <> struct Lattice<4> {  // D3Q343 = D1Q7 x D1Q7 x D1Q7
    static constexpr int D = 3, Q = 343;
    __host__ __device__ static constexpr int ex(int i) { return i % 7 - 3; }
    __host__ __device__ static constexpr int ey(int i) { return (i / 7) % 7 - 3; }
    __host__ __device__ static constexpr int ez(int i) { return i / 49 - 3; }
};

template <> struct Lattice<2> {
    static constexpr int D = 2, Q = 37;
    __host__ __device__ static constexpr int ex(int i) { return make_d2q37().x[i]; }
    __host__ __device__ static constexpr int ey(int i) { return make_d2q37().y[i]; }
    __host__ __device__ static constexpr int ez(int) { return 0; }
};

template <int LAT> __host__ __device__ constexpr int index_of(int ex, int ey, int ez)
{
    using L = Lattice<LAT>;
    for (int i = 0; i < L::Q; ++i)
        if (L::ex(i) == ex && L::ey(i) == ey && L::ez(i) == ez) return i;
    return -1;
}

template <int LAT> __host__ __device__ constexpr int e2_of(int i)
{
    using L = Lattice<LAT>;
    return L::ex(i) * L::ex(i) + L::ey(i) * L::ey(i) + L::ez(i) * L::ez(i);
}

// ---------------------------------------------------------------------------
// Population storage.  float: the value itself.  __half / __nv_bfloat16: the
// relative deviation from the rest equilibrium, d_i = f_i / w_i - 1 (the
// equilibrium at rho = 1, u = 0, T = 1 has d_i = 0), so the 11 (8) mantissa
// bits resolve the departure from rest rather than the weight's magnitude.
// All arithmetic stays float32; a value is decoded on load and encoded on
// store.
template <typename ST> struct Storage;
template <> struct Storage<__half> {
    __device__ static float decode(__half v, float w) { return fmaf(w, __half2float(v), w); }
    __device__ static __half encode(float f, float inv_w) { return __float2half_rn(fmaf(f, inv_w, -1.0f)); }
    __device__ static __half from_dev(float d) { return __float2half_rn(d); }
    __device__ static float to_dev(__half v) { return __half2float(v); }
};
template <> struct Storage<__nv_bfloat16> {
    __device__ static float decode(__nv_bfloat16 v, float w)
    {
        return fmaf(w, __bfloat162float(v), w);
    }
    __device__ static __nv_bfloat16 encode(float f, float inv_w)
    {
        return __float2bfloat16_rn(fmaf(f, inv_w, -1.0f));
    }
    __device__ static __nv_bfloat16 from_dev(float d) { return __float2bfloat16_rn(d); }
    __device__ static float to_dev(__nv_bfloat16 v) { return __bfloat162float(v); }
};

// Per-node reference storage (LBM_STORE_F16_NODE / BF16_NODE): the same
// 2-byte values, as distinct types so that every kernel knows at compile
// time whether a value is decoded with a reference record (ld, st_ref) and
// the plain 16-bit kernels carry no reference code.
struct NodeHalf {
    __half v;
};
struct NodeBf16 {
    __nv_bfloat16 v;
};
template <typename ST> struct NodeRef {
    static constexpr bool value = false;
    using elem = ST;
};
template <> struct NodeRef<NodeHalf> {
    static constexpr bool value = true;
    using elem = __half;
};
template <> struct NodeRef<NodeBf16> {
    static constexpr bool value = true;
    using elem = __nv_bfloat16;
};
template <typename N> struct NodeStorage {
    using E = typename NodeRef<N>::elem;
    __device__ static float decode(N v, float w) { return Storage<E>::decode(v.v, w); }
    __device__ static N encode(float f, float inv_w) { return N{Storage<E>::encode(f, inv_w)}; }
    __device__ static N from_dev(float d) { return N{Storage<E>::from_dev(d)}; }
};
template <> struct Storage<NodeHalf> : NodeStorage<NodeHalf> {};
template <> struct Storage<NodeBf16> : NodeStorage<NodeBf16> {};
using ::__ldcg;  // keep CUDA's overloads visible beside the two below
using ::__ldg;
__device__ __forceinline__ NodeHalf __ldg(const NodeHalf *a) { return NodeHalf{::__ldg(&a->v)}; }
__device__ __forceinline__ NodeBf16 __ldg(const NodeBf16 *a) { return NodeBf16{::__ldg(&a->v)}; }
__device__ __forceinline__ NodeHalf __ldcg(const NodeHalf *a) { return NodeHalf{::__ldcg(&a->v)}; }
__device__ __forceinline__ NodeBf16 __ldcg(const NodeBf16 *a) { return NodeBf16{::__ldcg(&a->v)}; }

// ---------------------------------------------------------------------------
// Kernel parameters (passed by value: they live in the constant bank, so the
// per-population weights become constant operands of the FMAs).

template <int Q, typename ST = float> struct Params {
    const ST *__restrict__ src;  // state, in the storage type
    ST *__restrict__ dst;
    const float *in0, *in1, *in2;
    float *out0, *out1, *out2;
    int *status;
    double *partials;
    const int64_t *nodes;
    int count;
    int64_t S, N;
    int X, Y, Z, pitch;
    int bc0, bc1, bc2;
    float r, r2, inv_r2, omega, nu_scale, cT, half_n, half_n_r2, inv_m;
    float w[Q], iw[Q];    // weights and their inverses (deviation storage)
    float wr[7], iwr[7];
    // lattice sums of the float weights: sum_i w_i, sum_i |e_i|^2 w_i and
    // sum_j (j-3)^2 wr_j (the deviation-space moment sums add these)
    float sw0 = 0.f, sw2 = 0.f, swr2 = 0.f;
    // Per-node reference storage (LBM_STORE_F16_NODE / BF16_NODE): records
    // (rho - 1, rho t / 2, rho r u_x, rho r u_y), t = T - 1, after the
    // populations of each buffer, and the per-population constants of the
    // reference R_i - 1 = (rho - 1) + e_x (rho r u_x) + e_y (rho r u_y)
    // + (|xi_i|^2 - D) rho t / 2 + kt2_i (rho t / 2)^2, kt2_i = (|xi|^4 -
    // 2 (D+2) |xi|^2 + D (D+2)) / 2 (the t^2 term of the Hermite
    // equilibrium with rho^2 t^2 standing for rho t^2), and
    // R_j^h - 1 = t (ha_j + t hb_j) (ref_dev).
    // (Null unless the storage type is a NodeRef one; kernels that fill a
    // Params field by field, like the ensemble's, leave them so.)
    const float4 *ref_src = nullptr;
    float4 *ref_dst = nullptr;
    static constexpr int NQ = (Q <= 49) ? Q : 1;
    float pex[NQ], pey[NQ], kmD[NQ], kt2[NQ];
    float ha[7], hb[7];
};

// t = T - 1 of a record, (rho t / 2) * 2 / rho with a correctly rounded
// reciprocal: the same bits wherever it is evaluated.
__device__ __forceinline__ float ref_t(float4 rc) { return (rc.y + rc.y) * __frcp_rn(1.0f + rc.x); }

// Deviation of the reference R from 1 for population `pop` (translational
// pop < Q, rotational pop - Q) under the record `rc`.  Writer and reader of a
// stored value both call this with the same record floats; the fused
// operations fix the rounding, so the reference cancels exactly.
template <int Q, typename ST>
__device__ __forceinline__ float ref_dev(const Params<Q, ST> &p, int pop, float4 rc, float ex, float ey,
                                         float kmd, float kt2)
{
    if (pop < Q) return fmaf(kt2, rc.y * rc.y, fmaf(kmd, rc.y, fmaf(ey, rc.w, fmaf(ex, rc.z, rc.x))));
    const int j = pop - Q;
    const float t = ref_t(rc);
    return t * fmaf(t, p.hb[j], p.ha[j]);
}
template <int Q, typename ST>
__device__ __forceinline__ float ref_dev(const Params<Q, ST> &p, int pop, float4 rc)
{
    if constexpr (Q <= 49) {
        if (pop < Q) return ref_dev(p, pop, rc, p.pex[pop], p.pey[pop], p.kmD[pop], p.kt2[pop]);
    }
    return ref_dev(p, pop, rc, 0.f, 0.f, 0.f, 0.f);
}

template <int Q, typename ST = float> Params<Q, ST> make_params(const Args &a)
{
    Params<Q, ST> p;
    p.src = static_cast<const ST *>(a.src);
    p.dst = static_cast<ST *>(a.dst);
    p.in0 = a.in0; p.in1 = a.in1; p.in2 = a.in2;
    p.out0 = a.out0; p.out1 = a.out1; p.out2 = a.out2;
    p.status = a.status;
    p.partials = a.partials;
    p.nodes = a.nodes;
    p.count = a.count;
    p.S = a.S;
    p.N = a.N;
    p.X = a.X; p.Y = a.Y; p.Z = a.Z; p.pitch = a.pitch;
    p.bc0 = a.bc[0]; p.bc1 = a.bc[1]; p.bc2 = a.bc[2];
    p.r = a.r;
    p.r2 = a.r * a.r;
    p.inv_r2 = 1.0f / (a.r * a.r);
    p.omega = a.omega;
    p.nu_scale = a.nu_scale;
    p.cT = a.cT;
    p.half_n_r2 = a.half_n_r2;
    p.half_n = a.half_n;
    p.inv_m = a.inv_m;
    for (int i = 0; i < Q; ++i) {
        p.w[i] = a.w[i];
        p.iw[i] = 1.0f / a.w[i];
    }
    for (int j = 0; j < 7; ++j) {
        p.wr[j] = a.wr[j];
        p.iwr[j] = 1.0f / a.wr[j];
    }
    double s0 = 0.0, s2 = 0.0, sr2 = 0.0;
    const D2Q37Table t37 = make_d2q37();
    for (int i = 0; i < Q; ++i) {
        // |e_i|^2 in each lattice's population order (the Lattice<> tables)
        int e2 = 0;
        if (Q == 37) e2 = t37.x[i] * t37.x[i] + t37.y[i] * t37.y[i];
        else
            for (int q = i, a3 = 0; a3 < 3 && (a3 == 0 || Q > (a3 == 1 ? 7 : 49)); ++a3, q /= 7)
                e2 += (q % 7 - 3) * (q % 7 - 3);
        s0 += (double)p.w[i];
        s2 += (double)e2 * (double)p.w[i];
    }
    for (int j = 0; j < 7; ++j) sr2 += (double)((j - 3) * (j - 3)) * (double)p.wr[j];
    p.sw0 = (float)s0;
    p.sw2 = (float)s2;
    p.swr2 = (float)sr2;
    constexpr bool node = NodeRef<ST>::value;
    p.ref_src = (node && a.src)
                    ? reinterpret_cast<const float4 *>(static_cast<const char *>(a.src) + a.ref_offset)
                    : nullptr;
    p.ref_dst = (node && a.dst) ? reinterpret_cast<float4 *>(static_cast<char *>(a.dst) + a.ref_offset)
                                : nullptr;
    const double rr = (double)a.r * (double)a.r;
    for (int i = 0; i < Params<Q, ST>::NQ; ++i) {
        int ex = 0, ey = 0;
        if (Q == 37) { ex = t37.x[i]; ey = t37.y[i]; }
        else if (Q <= 49) { ex = i % 7 - 3; ey = (Q == 49) ? i / 7 - 3 : 0; }
        p.pex[i] = (float)ex;
        p.pey[i] = (float)ey;
        const double si = rr * (ex * ex + ey * ey);  // |xi_i|^2
        p.kmD[i] = (float)(si - a.D);
        p.kt2[i] = (float)(0.5 * (si * si - 2.0 * (a.D + 2) * si + a.D * (a.D + 2)));
    }
    for (int j = 0; j < 7; ++j) {
        const double s2j = rr * (j - 3) * (j - 3);  // eta_j^2
        p.ha[j] = (float)(0.5 * (s2j - 1.0));
        p.hb[j] = (float)(0.125 * (s2j * s2j - 6.0 * s2j + 3.0));
    }
    return p;
}

// ---------------------------------------------------------------------------
// Boundary index: periodic wrap or copy (clamp to the edge node).  Offsets
// are at most 3, so one wrap suffices once the axis has >= 3 nodes.

__device__ __forceinline__ int bc_wrap(int x, int X, int bc)
{
    if (bc == 0) {
        if (X >= 3) {
            x = (x < 0) ? x + X : x;
            return (x >= X) ? x - X : x;
        }
        return ((x % X) + X) % X;
    }
    return min(max(x, 0), X - 1);
}

// Per-thread neighbour offsets (in floats) for shifts -3..+3 along each axis.
struct Offsets {
    int x[7], y[7], z[7];
    __device__ __forceinline__ int self() const { return z[3] + y[3] + x[3]; }
};

template <int D, int Q, typename ST>
__device__ __forceinline__ Offsets node_offsets(const Params<Q, ST> &p, int x, int y, int z)
{
    Offsets o;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        o.x[k] = bc_wrap(x + k - 3, p.X, p.bc0);
        o.y[k] = (D >= 2) ? bc_wrap(y + k - 3, p.Y, p.bc1) * p.pitch : 0;
        o.z[k] = (D >= 3) ? bc_wrap(z + k - 3, p.Z, p.bc2) * (p.pitch * p.Y) : 0;
    }
    return o;
}

// CG = 0: read-only path (the source buffer is never written during the
// launch).  CG = 1: L2-coherent loads, for kernels that read back what the
// same launch wrote (the persistent ensemble kernel).  CG = 2: plain
// generic loads (a state held in shared memory).
template <int CG = 0, int Q, typename ST>
__device__ __forceinline__ float ld(const Params<Q, ST> &p, int pop, int off)
{
    // 32-bit element index up to 49 populations; D3Q343 states exceed 2^32
    using Idx = typename std::conditional<(Q > 49), uint64_t, uint32_t>::type;
    const ST *a = p.src + ((Idx)pop * (Idx)p.S + (Idx)(uint32_t)off);
    ST v;
    if constexpr (CG == 2) v = *a;
    else if constexpr (CG == 1) v = __ldcg(a);
    else v = __ldg(a);
    if constexpr (std::is_same<ST, float>::value) return v;
    else {
        const float w = pop < Q ? p.w[pop] : p.wr[pop - Q];
        float f = Storage<ST>::decode(v, w);
        if constexpr (NodeRef<ST>::value) f = fmaf(w, ref_dev(p, pop, p.ref_src[(uint32_t)off]), f);
        return f;
    }
}
// Store relative to the record `rc` (per-node reference storage).
template <int Q, typename ST>
__device__ __forceinline__ void st_ref(const Params<Q, ST> &p, int pop, int off, float v, float4 rc)
{
    if constexpr (NodeRef<ST>::value) {
        const float iw = pop < Q ? p.iw[pop] : p.iwr[pop - Q];
        p.dst[(uint32_t)pop * (uint32_t)p.S + (uint32_t)off] =
            Storage<ST>::from_dev(fmaf(v, iw, -1.0f) - ref_dev(p, pop, rc));
    }
}
template <int Q, typename ST>
__device__ __forceinline__ void st(const Params<Q, ST> &p, int pop, int off, float v)
{
    using Idx = typename std::conditional<(Q > 49), uint64_t, uint32_t>::type;
    ST *a = p.dst + ((Idx)pop * (Idx)p.S + (Idx)(uint32_t)off);
    if constexpr (std::is_same<ST, float>::value) *a = v;
    else *a = Storage<ST>::encode(v, pop < Q ? p.iw[pop] : p.iwr[pop - Q]);
}

// ---------------------------------------------------------------------------
// Moments (Sec. V steps 3-4, Eq. T) of one node from its time-t populations.
// The velocity sums are taken per row/column first (partial sums by e_y and
// by e_x), which needs fewer operations than weighting every population.

struct Moments {
    float rho, ux, uy, uz, T, K, R;
    // the same in lattice units (velocities in units of r, no factors of r):
    // j_a = sum_i e_ia g_i, T_lat = T / r^2, E2_eq = sum_i |e_i|^2 g_i^eq
    float j[3], T_lat, E2_eq;
};

template <int D_, bool ROT, int Q, typename ST>
__device__ __forceinline__ Moments make_moments(const Params<Q, ST> &p, float rho, float jx,
                                                float jy, float jz, float e2, float R2);

template <int LAT, bool ROT, int Q, typename ST>
__device__ __forceinline__ Moments node_moments(const Params<Q, ST> &p, const float *g,
                                                const float *h)
{
    using L = Lattice<LAT>;
    float cs[7], rs[7], zs[7];  // sums over populations sharing e_x, e_y, e_z
    bool hc[7] = {}, hr[7] = {}, hz[7] = {};
#pragma unroll
    for (int k = 0; k < 7; ++k) cs[k] = rs[k] = zs[k] = 0.f;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const int a = L::ex(i) + 3, b = L::ey(i) + 3, c = L::ez(i) + 3;
        cs[a] = hc[a] ? cs[a] + g[i] : g[i];
        hc[a] = true;
        if (L::D >= 2) { rs[b] = hr[b] ? rs[b] + g[i] : g[i]; hr[b] = true; }
        if (L::D >= 3) { zs[c] = hz[c] ? zs[c] + g[i] : g[i]; hz[c] = true; }
    }
    // Opposite velocities are combined first (differences for the momentum,
    // sums for the energy), so a mirror-symmetric state gives exactly zero
    // momentum along that axis.
    float rho = cs[3], jx = 0.f, jy = 0.f, jz = 0.f, e2 = 0.f;
#pragma unroll
    for (int k = 1; k <= 3; ++k) {
        const float d = (float)k, dd = (float)(k * k);
        rho += cs[3 + k] + cs[3 - k];
        jx = fmaf(d, cs[3 + k] - cs[3 - k], jx);
        e2 = fmaf(dd, cs[3 + k] + cs[3 - k], e2);
        if (L::D >= 2) {
            jy = fmaf(d, rs[3 + k] - rs[3 - k], jy);
            e2 = fmaf(dd, rs[3 + k] + rs[3 - k], e2);
        }
        if (L::D >= 3) {
            jz = fmaf(d, zs[3 + k] - zs[3 - k], jz);
            e2 = fmaf(dd, zs[3 + k] + zs[3 - k], e2);
        }
    }
    float R2 = 0.f;
    if (ROT) {
#pragma unroll
        for (int k = 1; k <= 3; ++k) R2 = fmaf((float)(k * k), h[3 + k] + h[3 - k], R2);
    }
    return make_moments<L::D, ROT>(p, rho, jx, jy, jz, e2, R2);
}

// rho, u, T (Eq. T) from the lattice sums rho = sum g, j = sum e g,
// e2 = sum |e|^2 g and R2 = sum_j (j-3)^2 h_j.
template <int D_, bool ROT, int Q, typename ST>
__device__ __forceinline__ Moments make_moments(const Params<Q, ST> &p, float rho, float jx,
                                                float jy, float jz, float e2, float R2)
{
    constexpr int D = D_;
    Moments m;
    const float inv_rho = 1.0f / rho;
    m.rho = rho;
    m.j[0] = jx;
    m.j[1] = jy;
    m.j[2] = jz;
    m.ux = p.r * jx * inv_rho;
    m.uy = (D >= 2) ? p.r * jy * inv_rho : 0.f;
    m.uz = (D >= 3) ? p.r * jz * inv_rho : 0.f;
    m.K = 0.5f * p.r2 * e2;              // sum_i g_i xi_i^2 / 2
    m.R = ROT ? p.half_n_r2 * R2 : 0.f;  // sum_j (n/2) h_j eta_j^2
    // Eq. T evaluated in lattice units, then scaled once by r^2.  The factor
    // 2/(D+n) is applied as a division by (D+n)/2, which float represents
    // exactly: a rounded 2/(D+n) (0.4f for D+n = 5) would bias T, and with it
    // the total energy, by the same ~1e-8 every step.
    const float jj = (jx * jx + jy * jy + jz * jz) * inv_rho;  // rho u^2 / r^2
    if constexpr (sizeof(ST) < sizeof(float)) {
        // Reduced-precision storage: the temperature is recovered from the
        // total energy with the kinetic part subtracted in double precision,
        // where e2 - |j|^2 / rho cancels at high Mach.  Only that difference
        // needs double: |j|^2 of float components is exact in double, 1/rho
        // is the float reciprocal refined by one Newton step (relative error
        // ~1e-14), and the difference is formed by one fused multiply-add.
        // Everything after the cancellation keeps float's relative accuracy.
        // (GB300's FP64 pipe is slow: three double divisions per node held
        // the 16-bit step kernels to 56 % FP64-pipe utilisation.)
        double jjd = (double)jx * (double)jx;
        if (D >= 2) jjd = fma((double)jy, (double)jy, jjd);
        if (D >= 3) jjd = fma((double)jz, (double)jz, jjd);
        const double r0 = (double)inv_rho;
        const double inv_rho_d = fma(r0, fma(-(double)rho, r0, 1.0), r0);
        const float th = (float)fma(-jjd, inv_rho_d, (double)e2);  // 2 (K - rho u^2/2) / r^2
        m.T_lat = __fdiv_rn(0.5f * th * inv_rho + (ROT ? p.half_n * R2 : 0.f), p.cT);
    } else {
        m.T_lat = __fdiv_rn(0.5f * (e2 - jj) * inv_rho + (ROT ? p.half_n * R2 : 0.f), p.cT);
    }
    m.T = p.r2 * m.T_lat;
    m.E2_eq = jj + (float)D * rho * m.T_lat;  // rho (u^2 + D T) / r^2
    return m;
}

// Per-node coefficients of the 4th-order Hermite equilibrium written as a
// polynomial in c = xi.u with coefficients polynomial in s = |xi|^2:
//   g_i^eq / (w_i rho) = A0(s) + c A1(s) + c^2 A2(s) + c^3/6 + c^4/24,
// the collected form of sum_{k<=4} a^(k).H^(k)/k! (Sec. IV) with t = T - 1.
// Every coefficient is scaled by `scale` (omega rho in the step kernel).
struct EqCoef {
    float a00, a01, a02, a10, a11, a20, a21, k6, k24;
};

template <int D>
__device__ __forceinline__ EqCoef eq_coef(float T, float u2, float scale)
{
    const float t = T - 1.0f;
    EqCoef k;
    k.a00 = scale * (1.0f - 0.5f * u2 + 0.125f * u2 * u2 - 0.5f * t * D +
                     0.25f * t * (D + 2) * u2 + 0.125f * t * t * (D * (D + 2)));
    k.a01 = scale * (0.5f * t - 0.25f * t * u2 - 0.25f * t * t * (D + 2));
    k.a02 = scale * (0.125f * t * t);
    k.a10 = scale * (1.0f - 0.5f * u2 - 0.5f * t * (D + 2));
    k.a11 = scale * (0.5f * t);
    k.a20 = scale * (0.5f - 0.25f * u2 - 0.25f * t * (D + 4));
    k.a21 = scale * (0.25f * t);
    k.k6 = scale * (1.0f / 6.0f);
    k.k24 = scale * (1.0f / 24.0f);
    return k;
}

// The polynomial at +c and -c (a velocity and its opposite share s):
// P(+-c) = E +- O with E even and O odd in c.
__device__ __forceinline__ void eq_pair(const EqCoef &k, float c, float s, float &Pp, float &Pm)
{
    const float A0 = fmaf(s, fmaf(s, k.a02, k.a01), k.a00);
    const float A1 = fmaf(s, k.a11, k.a10);
    const float A2 = fmaf(s, k.a21, k.a20);
    const float c2 = c * c;
    const float E = fmaf(c2, fmaf(c2, k.k24, A2), A0);
    const float O = c * fmaf(c2, k.k6, A1);
    Pp = E + O;
    Pm = E - O;
}

__device__ __forceinline__ float eq_single(const EqCoef &k, float c, float s)
{
    float Pp, Pm;
    eq_pair(k, c, s, Pp, Pm);
    return Pp;
}

// h_j^eq / w_j on D1Q7 (Sec. IV): 1 + t(s-1)/2 + t^2 (s^2 - 6s + 3)/8, s = eta_j^2.
__device__ __forceinline__ float heq_poly(float t, float s)
{
    return 1.0f + 0.5f * t * (s - 1.0f) + 0.125f * t * t * (fmaf(s, s - 6.0f, 3.0f));
}

// Third-order upwind convection term (Sec. V) written for |nu|: with the
// upwind side chosen by the sign of nu, nu dF/dx = |nu| (F_uu - 6 F_u + 3 F_0
// + 2 F_d) / 6, where F_u, F_uu are the values one and two nodes upwind and
// F_d the value one node downwind.
__device__ __forceinline__ float upwind_abs(float anu, float fuu, float fu, float f0, float fd)
{
    return anu * ((fuu - 6.0f * fu + 3.0f * f0 + 2.0f * fd) * (1.0f / 6.0f));
}

// h^eq of one node with float32 moment corrections: the rounded weights make
// sum_j h_j^eq and sum_j eta_j^2 h_j^eq miss 1 and T by ~1e-8 every step, a
// drift that would accumulate; the defects are put back on the j = 3 (rest)
// and j = 2, 4 (+-r) entries, which leaves the odd moments untouched.  In
// exact arithmetic both corrections are zero.
template <int Q, typename ST>
__device__ __forceinline__ void heq_node(const Params<Q, ST> &p, float T, float T_lat, float *heq)
{
    const float t = T - 1.0f;
    float m0 = 0.f, m2 = 0.f;
#pragma unroll
    for (int j = 0; j < 7; ++j) {
        const int q = (j - 3) * (j - 3);
        heq[j] = p.wr[j] * heq_poly(t, p.r2 * (float)q);
        m0 += heq[j];
        if (q) m2 = fmaf((float)q, heq[j], m2);
    }
    const float b = 0.5f * (T_lat - m2);
    const float a = (1.0f - m0) - 2.0f * b;
    heq[3] += a;
    heq[2] += b;
    heq[4] += b;
}

// Rotational update (Eq. DisEvolSpaTiJ) of the 7 h_j at one node: upwind
// convection by u at Courant number u * nu_scale, BGK toward h^eq(T).
// (Issuing these neighbour loads right after the moments, before the
// translational work, measured 9 % slower on the 2048^2 workload.)
template <int D, int CG = 0, int Q, typename ST>
__device__ __forceinline__ void rot_advect(const Params<Q, ST> &p, const Offsets &o,
                                           const float *h, const Moments &m, float *adv)
{
#pragma unroll
    for (int j = 0; j < 7; ++j) adv[j] = 0.f;
    const float nu[3] = {m.ux * p.nu_scale, m.uy * p.nu_scale, m.uz * p.nu_scale};
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const int *oa = (a == 0) ? o.x : (a == 1) ? o.y : o.z;
        const int rest = o.self() - oa[3];
        const bool pos = nu[a] >= 0.0f;
        const int uu = rest + (pos ? oa[1] : oa[5]);  // two nodes upwind
        const int u1 = rest + (pos ? oa[2] : oa[4]);  // one node upwind
        const int d1 = rest + (pos ? oa[4] : oa[2]);  // one node downwind
        const float anu = fabsf(nu[a]);
#pragma unroll
        for (int j = 0; j < 7; ++j)
            adv[j] += upwind_abs(anu, ld<CG>(p, Q + j, uu), ld<CG>(p, Q + j, u1), h[j],
                                 ld<CG>(p, Q + j, d1));
    }
}

template <int Q, typename ST>
__device__ __forceinline__ void rot_store(const Params<Q, ST> &p, int self, const float *h,
                                          const Moments &m, const float *adv)
{
    float heq[7];
    heq_node(p, m.T, m.T_lat, heq);
    const float keep = 1.0f - p.omega;
#pragma unroll
    for (int j = 0; j < 7; ++j) st(p, Q + j, self, fmaf(keep, h[j], fmaf(p.omega, heq[j], -adv[j])));
}

// ---------------------------------------------------------------------------
// Load the time-t populations of one node.  STREAM: pull g_i(x) = ft_i(x - e_i).
// FD: g_i(x) = ft_i(x).

template <int LAT, bool ROT, int MODE, int CG = 0, int Q, typename ST>
__device__ __forceinline__ void load_node(const Params<Q, ST> &p, const Offsets &o, float *g,
                                          float *h)
{
    using L = Lattice<LAT>;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const int off = (MODE == 0)
                            ? o.z[3 - L::ez(i)] + o.y[3 - L::ey(i)] + o.x[3 - L::ex(i)]
                            : o.self();
        g[i] = ld<CG>(p, i, off);
    }
    if (ROT) {
#pragma unroll
        for (int j = 0; j < 7; ++j) h[j] = ld<CG>(p, L::Q + j, o.self());
    }
}

// FD transport of one translational population (Eq. DisEvolSpaTiI): the
// upwind side of each axis is fixed by the sign of e_ia, the Courant number
// is |e_ia| / m.
template <int LAT, int I, int CG = 0, int Q, typename ST>
__device__ __forceinline__ float fd_convect(const Params<Q, ST> &p, const Offsets &o, float g0)
{
    using L = Lattice<LAT>;
    float adv = 0.f;
    const int e[3] = {L::ex(I), L::ey(I), L::ez(I)};
#pragma unroll
    for (int a = 0; a < L::D; ++a) {
        if (e[a] == 0) continue;
        const int *oa = (a == 0) ? o.x : (a == 1) ? o.y : o.z;
        const int rest = o.self() - oa[3];
        const bool pos = e[a] > 0;
        const float anu = (float)(pos ? e[a] : -e[a]) * p.inv_m;
        adv += upwind_abs(anu, ld<CG>(p, I, rest + (pos ? oa[1] : oa[5])),
                          ld<CG>(p, I, rest + (pos ? oa[2] : oa[4])), g0,
                          ld<CG>(p, I, rest + (pos ? oa[4] : oa[2])));
    }
    return adv;
}

template <int LAT, int MODE, int I, int CG = 0, int Q, typename ST>
__device__ __forceinline__ float transport(const Params<Q, ST> &p, const Offsets &o, float g0)
{
    if constexpr (MODE == 1) return fd_convect<LAT, I, CG>(p, o, g0);
    return 0.f;
}

// Compile-time loop over the velocity pairs (I, Q-1-I), I below the centre.
template <int I, int N, typename F> __device__ __forceinline__ void static_for(F &&f)
{
    if constexpr (I < N) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, N>(f);
    }
}

// ---------------------------------------------------------------------------
// The fused step: moments -> equilibria -> BGK -> transport, one node per
// thread.  MODE 0 = STREAM (pull), 1 = FD (upwind forward Euler for g).
//
// Float32 moment corrections: with the weights rounded to float, the sums
// sum_i g_i^eq, sum_i e_i g_i^eq and sum_i |e_i|^2 g_i^eq miss rho, rho u/r
// and rho(u^2 + D T)/r^2 by ~1e-8 relative, a bias that would add up over
// thousands of steps.  The kernel accumulates these sums of omega g^eq as it
// writes the populations and puts the defects on the rest velocity and the
// 2D unit velocities +-1 along each axis, which are stored last: the
// momentum defect of axis a goes antisymmetrically onto +-1_a, the energy
// defect symmetrically onto all unit velocities, the rest keeps the mass.
// In exact arithmetic every correction is zero.

// Collision of one node's translational populations and their store
// (Eq. DisEvolI's BGK term, with the float32 corrections described above).
// `tr(I, g_I)` returns the transport term of population I (zero in STREAM
// mode, the upwind convection in FD mode).
template <int LAT, typename ST, typename Tr>
__device__ __forceinline__ void collide_store(const Params<Lattice<LAT>::Q, ST> &p, int self,
                                              const float *g, const Moments &m, Tr &&tr)
{
    using L = Lattice<LAT>;
    constexpr int Q = L::Q;
    constexpr int D = L::D;
    constexpr int C = (Q - 1) / 2;  // rest velocity
    const float u2 = m.ux * m.ux + m.uy * m.uy + m.uz * m.uz;
    const float om_rho = p.omega * m.rho;
    const EqCoef k = eq_coef<D>(m.T, u2, om_rho);  // omega rho g^eq / w_i
    const float keep = 1.0f - p.omega;
    const float ru[3] = {m.ux * p.r, m.uy * p.r, m.uz * p.r};
    float acc0 = 0.f, acc2 = 0.f;       // sums of omega g^eq and |e|^2 omega g^eq
    float accj[3] = {0.f, 0.f, 0.f};    // sums of e_a omega g^eq
    float qm[3] = {0.f, 0.f, 0.f}, qp[3] = {0.f, 0.f, 0.f};  // omega g^eq of -1_a, +1_a

    static_for<0, C>([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        constexpr int J = Q - 1 - I;
        constexpr int E2 = e2_of<LAT>(I);
        constexpr int e[3] = {L::ex(I), L::ey(I), L::ez(I)};
        float c = 0.f;
#pragma unroll
        for (int a = 0; a < D; ++a)
            if (e[a]) c = fmaf((float)e[a], ru[a], c);
        float Pp, Pm;
        eq_pair(k, c, p.r2 * (float)E2, Pp, Pm);
        const float qi = p.w[I] * Pp, qj = p.w[I] * Pm;  // w(-e) = w(e)
        const float sum = qi + qj, diff = qi - qj;
        acc0 += sum;
        acc2 = fmaf((float)E2, sum, acc2);
#pragma unroll
        for (int a = 0; a < D; ++a)
            if (e[a]) accj[a] = fmaf((float)e[a], diff, accj[a]);
        if constexpr (E2 == 1) {  // I is -1_a (the lower index of the pair)
            constexpr int ax = e[0] ? 0 : (e[1] ? 1 : 2);
            qm[ax] = qi;
            qp[ax] = qj;
        } else {
            st(p, I, self, fmaf(keep, g[I], qi) - tr(std::integral_constant<int, I>{}, g[I]));
            st(p, J, self, fmaf(keep, g[J], qj) - tr(std::integral_constant<int, J>{}, g[J]));
        }
    });
    const float q_c = p.w[C] * k.a00;  // rest velocity: c = 0, s = 0
    acc0 += q_c;
    const float d0 = om_rho - acc0;
    const float d2 = p.omega * m.E2_eq - acc2;
    const float b = d2 * (0.5f / (float)D);
    st(p, C, self, fmaf(keep, g[C], q_c + (d0 - d2)) - tr(std::integral_constant<int, C>{}, g[C]));
    static_for<0, D>([&](auto ac) {
        constexpr int A = decltype(ac)::value;
        constexpr int IM = index_of<LAT>(A == 0 ? -1 : 0, A == 1 ? -1 : 0, A == 2 ? -1 : 0);
        constexpr int IP = Q - 1 - IM;
        const float dm = 0.5f * (p.omega * m.j[A] - accj[A]);
        st(p, IM, self,
           fmaf(keep, g[IM], qm[A] + (b - dm)) - tr(std::integral_constant<int, IM>{}, g[IM]));
        st(p, IP, self,
           fmaf(keep, g[IP], qp[A] + (b + dm)) - tr(std::integral_constant<int, IP>{}, g[IP]));
    });
}

// (Two TMA variants were measured on the 2048^2 D2Q49 workload and dropped:
// staging each 128-node row tile's 84 source segments in shared memory with
// cp.async.bulk + an mbarrier ran 27 % slower -- blocks idle while their
// copies land and the smem per block halves the resident warps -- and
// cp.async.bulk.prefetch.L2 of rows 16..128 ahead ran 4..27 % slower.)
template <int LAT, bool ROT, int MODE, typename ST>
__global__ void LBM_STEP_BOUNDS k_step(const Params<Lattice<LAT>::Q, ST> p)
{
    using L = Lattice<LAT>;
    constexpr int Q = L::Q;
    constexpr int D = L::D;
    const int x = blockIdx.x * kBlockX + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= p.X) return;
    const Offsets o = node_offsets<D>(p, x, y, z);
    float g[Q], h[7];
    load_node<LAT, ROT, MODE>(p, o, g, h);
    const Moments m = node_moments<LAT, ROT>(p, g, h);
    if (!(m.rho > 0.f) || !(m.T > 0.f) || !(fabsf(m.T) < 3.0e38f)) atomicOr(p.status, 1);
    collide_store<LAT>(p, o.self(), g, m, [&](auto ic, float gi) {
        return transport<LAT, MODE, decltype(ic)::value>(p, o, gi);
    });
    if (ROT) {
        float adv[7];
        rot_advect<D>(p, o, h, m, adv);
        rot_store(p, o.self(), h, m, adv);
    }
}

// ---------------------------------------------------------------------------
// Initial state at equilibrium (pull pre-image in STREAM mode).

template <int LAT, bool ROT, int MODE, typename ST>
__device__ __forceinline__ void init_node(const Params<Lattice<LAT>::Q, ST> &p, int x, int y, int z)
{
    using L = Lattice<LAT>;
    const int self = (z * p.Y + y) * p.pitch + x;
    const float *rho_in = p.in0, *u_in = p.in1, *T_in = p.in2;
    constexpr bool is_node = NodeRef<ST>::value;
    float4 rc = make_float4(0.f, 0.f, 0.f, 0.f);
    if constexpr (is_node) {  // the node's reference: its own initial fields
        const int64_t node = ((int64_t)z * p.Y + y) * p.X + x;
        const float r0 = rho_in[node];
        rc = make_float4(r0 - 1.0f, 0.5f * (r0 * (T_in[node] - 1.0f)), r0 * (p.r * u_in[node]),
                         (L::D >= 2) ? r0 * (p.r * u_in[p.N + node]) : 0.f);
        p.ref_dst[self] = rc;
    }
#pragma unroll 1
    for (int i = 0; i < L::Q; ++i) {
        const int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
        int sx = x, sy = y, sz = z;
        if (MODE == 0) {
            sx = bc_wrap(x + ex, p.X, p.bc0);
            if (L::D >= 2) sy = bc_wrap(y + ey, p.Y, p.bc1);
            if (L::D >= 3) sz = bc_wrap(z + ez, p.Z, p.bc2);
        }
        const int64_t src = ((int64_t)sz * p.Y + sy) * p.X + sx;
        const float rho = rho_in[src];
        const float ux = u_in[src];
        const float uy = (L::D >= 2) ? u_in[p.N + src] : 0.f;
        const float uz = (L::D >= 3) ? u_in[2 * p.N + src] : 0.f;
        const float T = T_in[src];
        const EqCoef k = eq_coef<L::D>(T, ux * ux + uy * uy + uz * uz, rho);
        const float c = p.r * ((float)ex * ux + (float)ey * uy + (float)ez * uz);
        const float s = p.r2 * (float)(ex * ex + ey * ey + ez * ez);
        if constexpr (is_node) st_ref(p, i, self, p.w[i] * eq_single(k, c, s), rc);
        else st(p, i, self, p.w[i] * eq_single(k, c, s));
    }
    if (ROT) {
        const int64_t node = ((int64_t)z * p.Y + y) * p.X + x;
        float heq[7];
        const float Tn = T_in[node];
        heq_node(p, Tn, Tn * p.inv_r2, heq);
#pragma unroll
        for (int j = 0; j < 7; ++j) {
            if constexpr (is_node) st_ref(p, L::Q + j, self, heq[j], rc);
            else st(p, L::Q + j, self, heq[j]);
        }
    }
}

template <int LAT, bool ROT, int MODE, typename ST>
__global__ void __launch_bounds__(kBlockX) k_init(const Params<Lattice<LAT>::Q, ST> p)
{
    const int x = blockIdx.x * kBlockX + threadIdx.x;
    if (x >= p.X) return;
    init_node<LAT, ROT, MODE>(p, x, blockIdx.y, blockIdx.z);
}

// ---------------------------------------------------------------------------
// rho, u, T of the current state into unpadded caller arrays.

template <int LAT, bool ROT, int MODE, int CG = 0, typename ST>
__device__ __forceinline__ void moments_node(const Params<Lattice<LAT>::Q, ST> &p, int x, int y, int z)
{
    using L = Lattice<LAT>;
    const Offsets o = node_offsets<L::D>(p, x, y, z);
    float g[L::Q], h[7];
    load_node<LAT, ROT, MODE, CG>(p, o, g, h);
    const Moments m = node_moments<LAT, ROT>(p, g, h);
    const int64_t node = ((int64_t)z * p.Y + y) * p.X + x;
    p.out0[node] = m.rho;
    p.out1[node] = m.ux;
    if (L::D >= 2) p.out1[p.N + node] = m.uy;
    if (L::D >= 3) p.out1[2 * p.N + node] = m.uz;
    p.out2[node] = m.T;
}

template <int LAT, bool ROT, int MODE, typename ST>
__global__ void __launch_bounds__(kBlockX) k_moments(const Params<Lattice<LAT>::Q, ST> p)
{
    const int x = blockIdx.x * kBlockX + threadIdx.x;
    if (x >= p.X) return;
    moments_node<LAT, ROT, MODE>(p, x, blockIdx.y, blockIdx.z);
}

// ---------------------------------------------------------------------------
// Conservation diagnostics: per-block partial sums in double precision with a
// fixed grid and a fixed order (deterministic), finished by k_finalize.

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, off));
    return v;
}

template <int LAT, bool ROT, int MODE, typename ST>
__global__ void __launch_bounds__(kRedThreads) k_conserve(const Params<Lattice<LAT>::Q, ST> p)
{
    using L = Lattice<LAT>;
    double acc[kRedSlots] = {0, 0, 0, 0, 0, 0, 0, 0};  // mass, j[3], energy, hdev
    const int64_t stride = (int64_t)gridDim.x * kRedThreads;
    for (int64_t n = (int64_t)blockIdx.x * kRedThreads + threadIdx.x; n < p.N; n += stride) {
        const int x = (int)(n % p.X);
        const int y = (int)((n / p.X) % p.Y);
        const int z = (int)(n / ((int64_t)p.X * p.Y));
        const Offsets o = node_offsets<L::D>(p, x, y, z);
        float g[L::Q], h[7];
        load_node<LAT, ROT, MODE>(p, o, g, h);
        const Moments m = node_moments<LAT, ROT>(p, g, h);
        acc[0] += m.rho;
        acc[1] += (double)m.rho * m.ux;
        acc[2] += (double)m.rho * m.uy;
        acc[3] += (double)m.rho * m.uz;
        acc[4] += (double)m.K + (double)m.rho * m.R;
        if (ROT) {
            double sh = 0.0;
#pragma unroll
            for (int j = 0; j < 7; ++j) sh += h[j];
            acc[5] = fmax(acc[5], fabs(sh - 1.0));
        }
    }
    __shared__ double red[kRedSlots][kRedThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kRedSlots; ++k) {
        const double v = (k == 5) ? warp_max(acc[k]) : warp_sum(acc[k]);
        if (lane == 0) red[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < kRedSlots) {
        const int k = threadIdx.x;
        double v = 0.0;
        for (int w = 0; w < kRedThreads / 32; ++w) v = (k == 5) ? fmax(v, red[k][w]) : v + red[k][w];
        p.partials[(int64_t)blockIdx.x * kRedSlots + k] = v;
    }
}

// ---------------------------------------------------------------------------
// Canonical (unpadded) <-> internal (padded) population copies.

template <int LAT, bool ROT, typename ST>
__global__ void __launch_bounds__(kBlockX) k_get_state(const Params<Lattice<LAT>::Q, ST> p)
{
    using L = Lattice<LAT>;
    const int x = blockIdx.x * kBlockX + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= p.X) return;
    const int self = (z * p.Y + y) * p.pitch + x;
    const int64_t node = ((int64_t)z * p.Y + y) * p.X + x;
    for (int i = 0; i < L::Q; ++i) p.out0[(int64_t)i * p.N + node] = ld(p, i, self);
    if (ROT)
        for (int j = 0; j < 7; ++j) p.out1[(int64_t)j * p.N + node] = ld(p, L::Q + j, self);
}

// Sampled read-back: out0[k * (Q + Qr) + i] = population i of node nodes[k]
// (decoded to float), for checks at sizes too large to copy back whole.
template <int LAT, bool ROT, typename ST>
__global__ void k_sample(const Params<Lattice<LAT>::Q, ST> p)
{
    constexpr int Q = Lattice<LAT>::Q, QA = Q + (ROT ? 7 : 0);
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)p.count * QA) return;
    const int k = (int)(e / QA), i = (int)(e % QA);
    const int64_t node = p.nodes[k];
    const int x = (int)(node % p.X), y = (int)((node / p.X) % p.Y), z = (int)(node / ((int64_t)p.X * p.Y));
    const int self = (z * p.Y + y) * p.pitch + x;
    p.out0[e] = ld(p, i, self);
}

template <int LAT, bool ROT, typename ST>
__global__ void __launch_bounds__(kBlockX) k_set_state(const Params<Lattice<LAT>::Q, ST> p)
{
    using L = Lattice<LAT>;
    const int x = blockIdx.x * kBlockX + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= p.X) return;
    const int self = (z * p.Y + y) * p.pitch + x;
    const int64_t node = ((int64_t)z * p.Y + y) * p.X + x;
    if constexpr (NodeRef<ST>::value)
        p.ref_dst[self] = make_float4(0.f, 0.f, 0.f, 0.f);  // rest reference: R = 1
    for (int i = 0; i < L::Q; ++i) st(p, i, self, p.in0[(int64_t)i * p.N + node]);
    if (ROT)
        for (int j = 0; j < 7; ++j) st(p, L::Q + j, self, p.in1[(int64_t)j * p.N + node]);
}

#include "lbm_step_node.cuh"

// ---------------------------------------------------------------------------
// Host-side dispatch for one lattice.

// The D3Q343 step (lbm_d3q343.cu): STREAM transport only.
template <bool ROT, typename ST> cudaError_t launch_step_q343(const Args &a, cudaStream_t s);

template <int LAT, bool ROT, int MODE, typename ST>
cudaError_t launch_mode(Op op, const Args &a, cudaStream_t s)
{
    const auto p = make_params<Lattice<LAT>::Q, ST>(a);
    const dim3 block(kBlockX);
    const dim3 grid((a.X + kBlockX - 1) / kBlockX, a.Y, a.Z);
    switch (op) {
    case Op::Step:
        if constexpr (LAT == 4) {  // 343 populations: the two-pass kernel
            return launch_step_q343<ROT, ST>(a, s);
        } else if constexpr (NodeRef<ST>::value) {
            // per-node references: the deviation-space kernel (STREAM only)
            k_step_node<LAT, ROT, ST><<<grid, block, 0, s>>>(p);
        } else {
            k_step<LAT, ROT, MODE><<<grid, block, 0, s>>>(p);
        }
        break;
    case Op::Init: k_init<LAT, ROT, MODE><<<grid, block, 0, s>>>(p); break;
    case Op::Moments: k_moments<LAT, ROT, MODE><<<grid, block, 0, s>>>(p); break;
    case Op::Conserve: k_conserve<LAT, ROT, MODE><<<a.red_blocks, kRedThreads, 0, s>>>(p); break;
    case Op::GetState: k_get_state<LAT, ROT><<<grid, block, 0, s>>>(p); break;
    case Op::SetState: k_set_state<LAT, ROT><<<grid, block, 0, s>>>(p); break;
    case Op::Sample: {
        const int64_t n = (int64_t)a.count * (Lattice<LAT>::Q + (ROT ? 7 : 0));
        k_sample<LAT, ROT><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p);
        break;
    }
    }
    return cudaGetLastError();
}

template <int LAT, typename ST>
cudaError_t launch_storage(Op op, const Args &a, cudaStream_t s)
{
    const bool rot = a.Qr > 0;
    if constexpr (NodeRef<ST>::value) {  // STREAM on the 1-D and 2-D lattices only (host checks)
        if constexpr (LAT == 4) {
            return cudaErrorInvalidValue;
        } else {
            if (a.mode != 0) return cudaErrorInvalidValue;
            return rot ? launch_mode<LAT, true, 0, ST>(op, a, s) : launch_mode<LAT, false, 0, ST>(op, a, s);
        }
    } else {
        if (a.mode == 0 || LAT == 4)  // D3Q343 has no FD transport (the host rejects it)
            return rot ? launch_mode<LAT, true, 0, ST>(op, a, s) : launch_mode<LAT, false, 0, ST>(op, a, s);
        if constexpr (LAT != 4)
            return rot ? launch_mode<LAT, true, 1, ST>(op, a, s) : launch_mode<LAT, false, 1, ST>(op, a, s);
        return cudaErrorInvalidValue;
    }
}

template <int LAT>
cudaError_t launch_lattice(Op op, const Args &a, cudaStream_t s)
{
    switch (a.storage) {
    case 1: return launch_storage<LAT, __half>(op, a, s);
    case 2: return launch_storage<LAT, __nv_bfloat16>(op, a, s);
    case 3: return launch_storage<LAT, NodeHalf>(op, a, s);
    case 4: return launch_storage<LAT, NodeBf16>(op, a, s);
    default: return launch_storage<LAT, float>(op, a, s);
    }
}

}  // namespace lbm
