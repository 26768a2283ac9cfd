// Device code of the decoupled Hermite-expansion LBM (arXiv 1606.06107) for
// sm_103a.  Included by one translation unit per lattice, which instantiates
// the kernels for that lattice and defines its launch_<lattice>() entry.
//
// Memory layout in HBM: structure of arrays, population-major.  The state
// buffer holds Q_t translational arrays then Q_r rotational arrays, each of
// S = pitch * Y * Z floats, x fastest, rows padded to a multiple of 32 floats
// (128 bytes) so every row starts on a cache-line boundary.
//
// The step is memory bound: every population is read once and written once
// per step; all moments and equilibria live in registers.  One thread owns
// one node; a block is 128 consecutive x positions of one row.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "lbm_internal.h"

namespace lbm {

constexpr int kBlockX = 128;

// ---------------------------------------------------------------------------
// Velocity sets.  xi_i = r * e_i; order (ez, ey, ex) ascending.

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
template <> struct Lattice<2> {
    static constexpr int D = 2, Q = 37;
    __host__ __device__ static constexpr int ex(int i) { return make_d2q37().x[i]; }
    __host__ __device__ static constexpr int ey(int i) { return make_d2q37().y[i]; }
    __host__ __device__ static constexpr int ez(int) { return 0; }
};

// ---------------------------------------------------------------------------
// Kernel parameters (passed by value: they live in the constant bank, so the
// per-population weights become constant operands of the FMAs).

template <int Q> struct Params {
    const float *__restrict__ src;
    float *__restrict__ dst;
    const float *in0, *in1, *in2;
    float *out0, *out1, *out2;
    int *status;
    double *partials;
    int64_t S, N;
    int X, Y, Z, pitch;
    int bc0, bc1, bc2;
    float r, r2, omega, nu_scale, cT, half_n_r2, inv_m;
    float w[Q];
    float wr[7];
};

template <int Q> Params<Q> make_params(const Args &a)
{
    Params<Q> p;
    p.src = a.src;
    p.dst = a.dst;
    p.in0 = a.in0; p.in1 = a.in1; p.in2 = a.in2;
    p.out0 = a.out0; p.out1 = a.out1; p.out2 = a.out2;
    p.status = a.status;
    p.partials = a.partials;
    p.S = a.S;
    p.N = a.N;
    p.X = a.X; p.Y = a.Y; p.Z = a.Z; p.pitch = a.pitch;
    p.bc0 = a.bc[0]; p.bc1 = a.bc[1]; p.bc2 = a.bc[2];
    p.r = a.r;
    p.r2 = a.r * a.r;
    p.omega = a.omega;
    p.nu_scale = a.nu_scale;
    p.cT = a.cT;
    p.half_n_r2 = a.half_n_r2;
    p.inv_m = a.inv_m;
    for (int i = 0; i < Q; ++i) p.w[i] = a.w[i];
    for (int j = 0; j < 7; ++j) p.wr[j] = a.wr[j];
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

// Per-thread neighbour offsets for shifts -3..+3 along each axis (in floats).
struct Offsets {
    int x[7], y[7], z[7];
};

template <int D, int Q>
__device__ __forceinline__ Offsets node_offsets(const Params<Q> &p, int x, int y, int z)
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

// ---------------------------------------------------------------------------
// Moments (Sec. V steps 3-4, Eq. T) of one node from its time-t populations.

struct Moments {
    float rho, ux, uy, uz, T, K, R;
};

template <int LAT, bool ROT, int Q>
__device__ __forceinline__ Moments node_moments(const Params<Q> &p, const float *g,
                                                const float *h)
{
    using L = Lattice<LAT>;
    float rho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f, e2 = 0.f;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
        rho += g[i];
        if (ex) jx = fmaf((float)ex, g[i], jx);
        if (L::D >= 2 && ey) jy = fmaf((float)ey, g[i], jy);
        if (L::D >= 3 && ez) jz = fmaf((float)ez, g[i], jz);
        const int ee = ex * ex + ey * ey + ez * ez;
        if (ee) e2 = fmaf((float)ee, g[i], e2);
    }
    float R2 = 0.f;
    if (ROT) {
#pragma unroll
        for (int j = 0; j < 7; ++j) {
            const int q = (j - 3) * (j - 3);
            if (q) R2 = fmaf((float)q, h[j], R2);
        }
    }
    Moments m;
    const float inv_rho = 1.0f / rho;
    m.rho = rho;
    m.ux = p.r * jx * inv_rho;
    m.uy = (L::D >= 2) ? p.r * jy * inv_rho : 0.f;
    m.uz = (L::D >= 3) ? p.r * jz * inv_rho : 0.f;
    m.K = 0.5f * p.r2 * e2;          // sum_i g_i xi_i^2 / 2
    m.R = ROT ? p.half_n_r2 * R2 : 0.f;  // sum_j (n/2) h_j eta_j^2
    const float u2 = m.ux * m.ux + m.uy * m.uy + m.uz * m.uz;
    m.T = p.cT * (m.K * inv_rho + m.R - 0.5f * u2);
    return m;
}

// Per-node coefficients of the 4th-order Hermite equilibrium written as a
// polynomial in c = xi.u with coefficients polynomial in s = |xi|^2:
//   g_i^eq / (w_i rho) = A0(s) + c A1(s) + c^2 A2(s) + c^3/6 + c^4/24,
// the collected form of sum_{k<=4} a^(k).H^(k)/k! (Sec. IV) with t = T - 1.
struct EqCoef {
    float a00, a01, a02, a10, a11, a20, a21;
};

template <int D>
__device__ __forceinline__ EqCoef eq_coef(float T, float u2)
{
    const float t = T - 1.0f;
    EqCoef k;
    k.a00 = 1.0f - 0.5f * u2 + 0.125f * u2 * u2 - 0.5f * t * D + 0.25f * t * (D + 2) * u2 +
            0.125f * t * t * (D * (D + 2));
    k.a01 = 0.5f * t - 0.25f * t * u2 - 0.25f * t * t * (D + 2);
    k.a02 = 0.125f * t * t;
    k.a10 = 1.0f - 0.5f * u2 - 0.5f * t * (D + 2);
    k.a11 = 0.5f * t;
    k.a20 = 0.5f - 0.25f * u2 - 0.25f * t * (D + 4);
    k.a21 = 0.25f * t;
    return k;
}

__device__ __forceinline__ float eq_poly(const EqCoef &k, float c, float s)
{
    const float A0 = fmaf(s, fmaf(s, k.a02, k.a01), k.a00);
    const float A1 = fmaf(s, k.a11, k.a10);
    const float A2 = fmaf(s, k.a21, k.a20);
    float P = fmaf(c, 1.0f / 24.0f, 1.0f / 6.0f);
    P = fmaf(c, P, A2);
    P = fmaf(c, P, A1);
    return fmaf(c, P, A0);
}

// h_j^eq / w_j on D1Q7 (Sec. IV): 1 + t(s-1)/2 + t^2 (s^2 - 6s + 3)/8, s = eta_j^2.
__device__ __forceinline__ float heq_poly(float t, float s)
{
    return 1.0f + 0.5f * t * (s - 1.0f) + 0.125f * t * t * (fmaf(s, s - 6.0f, 3.0f));
}

// Third-order upwind convection term nu * dF/dx (Sec. V): the backward
// stencil for nu >= 0, the forward one for nu < 0.
__device__ __forceinline__ float stencil_back(float fm2, float fm1, float f0, float fp1)
{
    return (fm2 - 6.0f * fm1 + 3.0f * f0 + 2.0f * fp1) * (1.0f / 6.0f);
}
__device__ __forceinline__ float stencil_fwd(float fm1, float f0, float fp1, float fp2)
{
    return (-fp2 + 6.0f * fp1 - 3.0f * f0 - 2.0f * fm1) * (1.0f / 6.0f);
}
__device__ __forceinline__ float upwind(float nu, float fm2, float fm1, float f0, float fp1,
                                        float fp2)
{
    return nu >= 0.0f ? nu * stencil_back(fm2, fm1, f0, fp1) : nu * stencil_fwd(fm1, f0, fp1, fp2);
}

// Rotational update (Eq. DisEvolSpaTiJ) of the 7 h_j at one node: upwind
// convection by u at Courant number u * nu_scale, BGK toward h^eq(T).
template <int D, int Q>
__device__ __forceinline__ void rot_update(const Params<Q> &p, const Offsets &o,
                                           const float *h, const Moments &m)
{
    const int64_t self = (int64_t)o.z[3] + o.y[3] + o.x[3];
    const float t = m.T - 1.0f;
    const float nux = m.ux * p.nu_scale, nuy = m.uy * p.nu_scale, nuz = m.uz * p.nu_scale;
#pragma unroll
    for (int j = 0; j < 7; ++j) {
        const float *F = p.src + (int64_t)(Q + j) * p.S;
        const float s = p.r2 * (float)((j - 3) * (j - 3));
        const float heq = p.wr[j] * heq_poly(t, s);
        const int rowz = o.z[3] + o.y[3];
        float adv = upwind(nux, __ldg(F + rowz + o.x[1]), __ldg(F + rowz + o.x[2]), h[j],
                           __ldg(F + rowz + o.x[4]), __ldg(F + rowz + o.x[5]));
        if (D >= 2) {
            const int colz = o.z[3] + o.x[3];
            adv += upwind(nuy, __ldg(F + colz + o.y[1]), __ldg(F + colz + o.y[2]), h[j],
                          __ldg(F + colz + o.y[4]), __ldg(F + colz + o.y[5]));
        }
        if (D >= 3) {
            const int rowy = o.y[3] + o.x[3];
            adv += upwind(nuz, __ldg(F + rowy + o.z[1]), __ldg(F + rowy + o.z[2]), h[j],
                          __ldg(F + rowy + o.z[4]), __ldg(F + rowy + o.z[5]));
        }
        p.dst[(int64_t)(Q + j) * p.S + self] = h[j] - adv - p.omega * (h[j] - heq);
    }
}

// ---------------------------------------------------------------------------
// Load the time-t populations of one node.  STREAM: pull g_i(x) = ft_i(x - e_i).
// FD: g_i(x) = ft_i(x).

template <int LAT, bool ROT, int MODE, int Q>
__device__ __forceinline__ void load_node(const Params<Q> &p, const Offsets &o, float *g,
                                          float *h)
{
    using L = Lattice<LAT>;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const int off = (MODE == 0)
                            ? o.z[3 - L::ez(i)] + o.y[3 - L::ey(i)] + o.x[3 - L::ex(i)]
                            : o.z[3] + o.y[3] + o.x[3];
        g[i] = __ldg(p.src + (int64_t)i * p.S + off);
    }
    if (ROT) {
        const int self = o.z[3] + o.y[3] + o.x[3];
#pragma unroll
        for (int j = 0; j < 7; ++j) h[j] = __ldg(p.src + (int64_t)(L::Q + j) * p.S + self);
    }
}

// ---------------------------------------------------------------------------
// The fused step: moments -> equilibria -> BGK -> transport, one node per
// thread.  MODE 0 = STREAM (pull), 1 = FD (upwind forward Euler for g).

template <int LAT, bool ROT, int MODE>
__global__ void __launch_bounds__(kBlockX) k_step(const Params<Lattice<LAT>::Q> p)
{
    using L = Lattice<LAT>;
    constexpr int Q = L::Q;
    const int x = blockIdx.x * kBlockX + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= p.X) return;
    const Offsets o = node_offsets<L::D>(p, x, y, z);
    float g[Q], h[7];
    load_node<LAT, ROT, MODE>(p, o, g, h);
    const Moments m = node_moments<LAT, ROT>(p, g, h);
    if (!(m.rho > 0.f) || !(m.T > 0.f) || !(fabsf(m.T) < 3.0e38f)) atomicOr(p.status, 1);

    const float u2 = m.ux * m.ux + m.uy * m.uy + m.uz * m.uz;
    const EqCoef k = eq_coef<L::D>(m.T, u2);
    const float om_rho = p.omega * m.rho;
    const float keep = 1.0f - p.omega;
    const float rux = m.ux * p.r, ruy = m.uy * p.r, ruz = m.uz * p.r;
    const int self = o.z[3] + o.y[3] + o.x[3];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
        const float c = (float)ex * rux + (float)ey * ruy + (float)ez * ruz;
        const float s = p.r2 * (float)(ex * ex + ey * ey + ez * ez);
        const float P = eq_poly(k, c, s);
        float out = fmaf(om_rho * p.w[i], P, keep * g[i]);
        if (MODE == 1) {  // Eq. DisEvolSpaTiI: - dt xi_i . grad g_i, Courant e_ia / m
            const float *F = p.src + (int64_t)i * p.S;
            if (ex) {
                const int row = o.z[3] + o.y[3];
                const float nu = (float)ex * p.inv_m;
                out -= nu * ((ex > 0) ? stencil_back(__ldg(F + row + o.x[1]), __ldg(F + row + o.x[2]),
                                                     g[i], __ldg(F + row + o.x[4]))
                                      : stencil_fwd(__ldg(F + row + o.x[2]), g[i],
                                                    __ldg(F + row + o.x[4]), __ldg(F + row + o.x[5])));
            }
            if (L::D >= 2 && ey) {
                const int col = o.z[3] + o.x[3];
                const float nu = (float)ey * p.inv_m;
                out -= nu * ((ey > 0) ? stencil_back(__ldg(F + col + o.y[1]), __ldg(F + col + o.y[2]),
                                                     g[i], __ldg(F + col + o.y[4]))
                                      : stencil_fwd(__ldg(F + col + o.y[2]), g[i],
                                                    __ldg(F + col + o.y[4]), __ldg(F + col + o.y[5])));
            }
            if (L::D >= 3 && ez) {
                const int rw = o.y[3] + o.x[3];
                const float nu = (float)ez * p.inv_m;
                out -= nu * ((ez > 0) ? stencil_back(__ldg(F + rw + o.z[1]), __ldg(F + rw + o.z[2]),
                                                     g[i], __ldg(F + rw + o.z[4]))
                                      : stencil_fwd(__ldg(F + rw + o.z[2]), g[i],
                                                    __ldg(F + rw + o.z[4]), __ldg(F + rw + o.z[5])));
            }
        }
        p.dst[(int64_t)i * p.S + self] = out;
    }
    if (ROT) rot_update<L::D>(p, o, h, m);
}

// ---------------------------------------------------------------------------
// Initial state at equilibrium (pull pre-image in STREAM mode).

template <int LAT, bool ROT, int MODE>
__global__ void __launch_bounds__(kBlockX) k_init(const Params<Lattice<LAT>::Q> p)
{
    using L = Lattice<LAT>;
    const int x = blockIdx.x * kBlockX + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= p.X) return;
    const int self = (z * p.Y + y) * p.pitch + x;
    const float *rho_in = p.in0, *u_in = p.in1, *T_in = p.in2;
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
        const EqCoef k = eq_coef<L::D>(T, ux * ux + uy * uy + uz * uz);
        const float c = p.r * ((float)ex * ux + (float)ey * uy + (float)ez * uz);
        const float s = p.r2 * (float)(ex * ex + ey * ey + ez * ez);
        p.dst[(int64_t)i * p.S + self] = p.w[i] * rho * eq_poly(k, c, s);
    }
    if (ROT) {
        const int64_t node = ((int64_t)z * p.Y + y) * p.X + x;
        const float t = T_in[node] - 1.0f;
#pragma unroll
        for (int j = 0; j < 7; ++j) {
            const float s = p.r2 * (float)((j - 3) * (j - 3));
            p.dst[(int64_t)(L::Q + j) * p.S + self] = p.wr[j] * heq_poly(t, s);
        }
    }
}

// ---------------------------------------------------------------------------
// rho, u, T of the current state into unpadded caller arrays.

template <int LAT, bool ROT, int MODE>
__global__ void __launch_bounds__(kBlockX) k_moments(const Params<Lattice<LAT>::Q> p)
{
    using L = Lattice<LAT>;
    const int x = blockIdx.x * kBlockX + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= p.X) return;
    const Offsets o = node_offsets<L::D>(p, x, y, z);
    float g[L::Q], h[7];
    load_node<LAT, ROT, MODE>(p, o, g, h);
    const Moments m = node_moments<LAT, ROT>(p, g, h);
    const int64_t node = ((int64_t)z * p.Y + y) * p.X + x;
    p.out0[node] = m.rho;
    p.out1[node] = m.ux;
    if (L::D >= 2) p.out1[p.N + node] = m.uy;
    if (L::D >= 3) p.out1[2 * p.N + node] = m.uz;
    p.out2[node] = m.T;
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

template <int LAT, bool ROT, int MODE>
__global__ void __launch_bounds__(kRedThreads) k_conserve(const Params<Lattice<LAT>::Q> p)
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
            float sh = 0.f;
#pragma unroll
            for (int j = 0; j < 7; ++j) sh += h[j];
            acc[5] = fmax(acc[5], fabs((double)sh - 1.0));
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

template <int LAT, bool ROT>
__global__ void __launch_bounds__(kBlockX) k_get_state(const Params<Lattice<LAT>::Q> p)
{
    using L = Lattice<LAT>;
    const int x = blockIdx.x * kBlockX + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= p.X) return;
    const int64_t self = ((int64_t)z * p.Y + y) * p.pitch + x;
    const int64_t node = ((int64_t)z * p.Y + y) * p.X + x;
    for (int i = 0; i < L::Q; ++i) p.out0[(int64_t)i * p.N + node] = p.src[(int64_t)i * p.S + self];
    if (ROT)
        for (int j = 0; j < 7; ++j)
            p.out1[(int64_t)j * p.N + node] = p.src[(int64_t)(L::Q + j) * p.S + self];
}

template <int LAT, bool ROT>
__global__ void __launch_bounds__(kBlockX) k_set_state(const Params<Lattice<LAT>::Q> p)
{
    using L = Lattice<LAT>;
    const int x = blockIdx.x * kBlockX + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= p.X) return;
    const int64_t self = ((int64_t)z * p.Y + y) * p.pitch + x;
    const int64_t node = ((int64_t)z * p.Y + y) * p.X + x;
    for (int i = 0; i < L::Q; ++i) p.dst[(int64_t)i * p.S + self] = p.in0[(int64_t)i * p.N + node];
    if (ROT)
        for (int j = 0; j < 7; ++j)
            p.dst[(int64_t)(L::Q + j) * p.S + self] = p.in1[(int64_t)j * p.N + node];
}

// ---------------------------------------------------------------------------
// Host-side dispatch for one lattice.

template <int LAT, bool ROT, int MODE>
cudaError_t launch_mode(Op op, const Args &a, cudaStream_t s)
{
    const auto p = make_params<Lattice<LAT>::Q>(a);
    const dim3 block(kBlockX);
    const dim3 grid((a.X + kBlockX - 1) / kBlockX, a.Y, a.Z);
    switch (op) {
    case Op::Step: k_step<LAT, ROT, MODE><<<grid, block, 0, s>>>(p); break;
    case Op::Init: k_init<LAT, ROT, MODE><<<grid, block, 0, s>>>(p); break;
    case Op::Moments: k_moments<LAT, ROT, MODE><<<grid, block, 0, s>>>(p); break;
    case Op::Conserve: k_conserve<LAT, ROT, MODE><<<a.red_blocks, kRedThreads, 0, s>>>(p); break;
    case Op::GetState: k_get_state<LAT, ROT><<<grid, block, 0, s>>>(p); break;
    case Op::SetState: k_set_state<LAT, ROT><<<grid, block, 0, s>>>(p); break;
    }
    return cudaGetLastError();
}

template <int LAT>
cudaError_t launch_lattice(Op op, const Args &a, cudaStream_t s)
{
    const bool rot = a.Qr > 0;
    if (a.mode == 0)
        return rot ? launch_mode<LAT, true, 0>(op, a, s) : launch_mode<LAT, false, 0>(op, a, s);
    return rot ? launch_mode<LAT, true, 1>(op, a, s) : launch_mode<LAT, false, 1>(op, a, s);
}

}  // namespace lbm
