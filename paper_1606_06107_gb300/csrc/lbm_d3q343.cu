// Kernel instantiations for the D3Q343 lattice (D1Q7 x D1Q7 x D1Q7) and its
// two-pass STREAM step.
//
// 343 populations do not fit in registers, so the step reads its pulled
// populations twice: a first pass accumulates rho, j and sum |e|^2 g (row
// sums by (e_y, e_z), column sums by e_x), a second pass re-reads each value
// (from a shared-memory stash for the first planes with 16-bit storage, else
// from L1/L2: a 128-node block touches 343 x 128 x 4 B = 175 KB between the
// two reads) and writes its post-collision value (with 16-bit storage as a
// deviation computed from the stored deviation, below).  The second pass walks the
// e_z planes in reverse, so that it starts on the lines the first pass loaded
// last, which are the ones still in L1 (7 % faster with float storage, 1 %
// with f16).  The rest and the six unit
// velocities are stored last with the float32 moment corrections, as in the
// one- and two-dimensional kernels.  Element indices are 64-bit (the state
// of a 384^3 grid holds 2 x 10^10 values).
#include <atomic>

#include "lbm_step.cuh"

namespace lbm {
namespace {

constexpr int kQ343 = 343;

// Resident blocks per SM the register allocation must allow.  Left free the
// compiler takes 185-207 registers (2 blocks of 4 warps); 3 blocks (at most
// 170 registers, 0-60 bytes of spill) measured 13 % (n = 0) and 7 % (n = 4)
// faster on the 384^3 f16 blast; 4 blocks (128 registers, at most 4 stash
// planes in the shared memory) are slower: with the row quartic and no
// spills 34.7 / 45.8 ms with 4 planes and 33.9 / 43.0 with 3, against 28.0
// / 32.0 at 3 blocks with 6.
#ifndef LBM_Q343_MIN_BLOCKS
#define LBM_Q343_MIN_BLOCKS 3
#endif
// Shared-memory stash of the first pass's raw values for the e_z planes
// c < NS, which the second pass (walking the planes in reverse) reaches
// last, when L1 has long evicted them.  16-bit values take 12.5 KB per plane
// per 128-thread block.  With the deviation-form pass 2 below, on the 384^3
// f16 blast (ms per step, n = 0 / n = 4): with the row quartic 5 planes
// 28.1 / 33.4, 6 planes 28.0 / 32.0; before it 4 planes 32.6 / 36.2, 5
// planes 31.0 / 35.0, 6 planes 32.6 / 36.5 (with the weight-table pass 2 6 planes
// had been best: none 36.2 / 42.2, 4 35.2 / 41.3, 5 33.3 / 39.4, 6 33.0 /
// 38.8, all 7 at 2 blocks per SM 43.9 / 46.9).  Float storage gained nothing
// from 2 planes.  The second pass decodes the same stored bits, so the depth
// does not change results.
#ifndef LBM_Q343_STASH_HALF
#define LBM_Q343_STASH_HALF 6
#endif
#ifndef LBM_Q343_STASH_FLOAT
#define LBM_Q343_STASH_FLOAT 0
#endif
// Threads per block of the step (x positions of one row).  Measured on the
// 384^3 f16 blast (ms per step, n = 0 / n = 4): 128 threads at 3 blocks per
// SM 34.1 / 39.8; 64 at 6 36.6 / 42.4; 64 at 7 with 5 stash planes 49.6 /
// 55.7; 64 at 8 with 4 planes 42.7 / 49.8; 32 at 12 47.5 / 55.0.  Narrower
// blocks share fewer of the pulled rows' lines in L1.
#ifndef LBM_Q343_BLOCK
#define LBM_Q343_BLOCK 128
#endif
constexpr int kQ343Block = LBM_Q343_BLOCK;

template <typename ST> struct StashPlanes {
    static constexpr int value = std::is_same<ST, float>::value ? LBM_Q343_STASH_FLOAT : LBM_Q343_STASH_HALF;
};
template <typename ST> constexpr size_t stash_bytes() { return (size_t)StashPlanes<ST>::value * 49 * kQ343Block * sizeof(ST); }

template <int Q, typename ST>
__device__ __forceinline__ float decode_pop(const Params<Q, ST> &p, int pop, ST v)
{
    if constexpr (std::is_same<ST, float>::value) return v;
    else return Storage<ST>::decode(v, p.w[pop]);
}

// Population i of the node at in-population offset off (64-bit element
// index: the state of a 384^3 grid holds 2 x 10^10 values).
template <typename ST>
__device__ __forceinline__ ST q343_load(const Params<kQ343, ST> &p, int i, int off)
{
    return __ldg(p.src + ((uint64_t)i * (uint64_t)p.S + (uint64_t)(uint32_t)off));
}
template <typename ST>
__device__ __forceinline__ void q343_store(const Params<kQ343, ST> &p, int i, int self, float v)
{
    ST val;
    if constexpr (std::is_same<ST, float>::value) val = v;
    else val = Storage<ST>::encode(v, p.iw[i]);
    p.dst[(uint64_t)i * (uint64_t)p.S + (uint32_t)self] = val;
}

// Pass 2 with 16-bit deviation storage, d_i = f_i / w_i - 1, runs on the
// deviations with the weights factored.  D3Q343 = D1Q7^3, so w_i = w_a w_b
// w_c.  The e_z planes c are a run-time loop, so a table lookup w[i] (or
// 1 / w[i]) is a run-time-indexed parameter load for every population; here
// the in-plane factors w_a w_b, w_a w_b e_x and w_a w_b e_x^2 (compile-time
// indices inside the unrolled row) are immediate operands of the row sums and
// the plane factor w_c multiplies the plane sums once.  The collision
// f* = (1 - omega) g + omega g^eq becomes d* = (1 - omega) d + (P - omega)
// with P = omega rho g^eq / w, so no value is decoded to f or encoded back.
// The equilibrium along each row is evaluated as a quartic in e_x (below),
// 6 operations per pair of populations e_x = +-k instead of a full
// polynomial evaluation for each.
// Measured on the 384^3 f16 blast (ms per step, n = 0 / n = 4, 6 stash
// planes): 33.7 / 40.1 with the weight table, 32.6 / 36.5 in this form with
// the equilibrium evaluated per population, 28.0 / 32.0 with the row
// quartic (fewer registers: 8 bytes of spill instead of 176); the
// same treatment of pass 1 (weighted deviation sums scaled by w_c per row)
// took 35.4 / 45.0 alone and 36.5 / 40.2 with both (more registers, spills);
// with 5 stash planes, 30.8 / 36.2 with both against 31.1 / 35.2 for pass 2
// alone.  One body per pass with the stash choice a run-time predicate
// (half the code, against the instruction-cache misses) instead of the two
// compile-time bodies per pass: 31.0 / 35.9 (pass 1), 36.7 / 37.8 (pass 2),
// 35.5 / 38.0 (both) against 30.9 / 35.0.
#ifndef LBM_Q343_DEV
#define LBM_Q343_DEV 1
#endif
struct Q343Weights {
    float w2[49];    // w_a w_b, index b * 7 + a
    float w2x[49];   // w_a w_b e_x
    float w2x2[49];  // w_a w_b e_x^2
    float wc[7];     // w_c
    float iw_rest, iw_unit;  // 1 / w of the rest velocity and of the unit velocities
};
template <typename ST> struct Q343Dev {
    static constexpr bool value = LBM_Q343_DEV && !std::is_same<ST, float>::value;
};
template <typename ST>
__device__ __forceinline__ void q343_store_dev(const Params<kQ343, ST> &p, int i, int self, float d)
{
    p.dst[(uint64_t)i * (uint64_t)p.S + (uint32_t)self] = Storage<ST>::from_dev(d);
}

// The five sums of pass 1: rho, j and sum_i |e_i|^2 g_i (lattice units).
struct Q343Sums {
    float rho, jx, jy, jz, e2;
};

// Pass 1 of one node: moments of the pulled populations g_i(x) = ft_i(x - e_i).
// The raw values of the e_z planes c < NS are kept in the stash for pass 2.
template <int NS, typename ST>
__device__ __forceinline__ Q343Sums q343_sums(const Params<kQ343, ST> &p, const Offsets &o, int z, ST *stash)
{
    const int plane = p.pitch * p.Y;
    float cs[7];
#pragma unroll
    for (int a = 0; a < 7; ++a) cs[a] = 0.f;
    float rho = 0.f, jy = 0.f, jz = 0.f, e2yz = 0.f;
    // e_y is unrolled so that each e_z plane issues its 49 loads at once
    auto plane1 = [&](auto keep, int c) {
        constexpr bool KEEP = decltype(keep)::value;
        const int zo = bc_wrap(z - (c - 3), p.Z, p.bc2) * plane;
#pragma unroll
        for (int b = 0; b < 7; ++b) {
            const int row = zo + o.y[6 - b];
            float rsum = 0.f;
#pragma unroll
            for (int a = 0; a < 7; ++a) {
                const int i = (c * 7 + b) * 7 + a;
                const ST v = q343_load(p, i, row + o.x[6 - a]);
                if constexpr (KEEP) stash[i * kQ343Block + threadIdx.x] = v;
                const float g = decode_pop(p, i, v);
                cs[a] += g;
                rsum += g;
            }
            const float db = (float)(b - 3), dc = (float)(c - 3);
            rho += rsum;
            jy = fmaf(db, rsum, jy);
            jz = fmaf(dc, rsum, jz);
            e2yz = fmaf(db * db + dc * dc, rsum, e2yz);
        }
    };
    for (int c = 0; c < 7; ++c) {
        if (c < NS) plane1(std::true_type{}, c);
        else plane1(std::false_type{}, c);
    }
    float jx = 0.f, e2 = e2yz;
#pragma unroll
    for (int k = 1; k <= 3; ++k) {
        jx = fmaf((float)k, cs[3 + k] - cs[3 - k], jx);
        e2 = fmaf((float)(k * k), cs[3 + k] + cs[3 - k], e2);
    }
    return Q343Sums{rho, jx, jy, jz, e2};
}

// The equilibrium polynomial along a row.  With e_y, e_z fixed, c = xi . u
// = C0 + e_x v and s = |xi|^2 = S0 + r^2 e_x^2, so P = A0(s) + A1(s) c +
// A2(s) c^2 + k6 c^3 + k24 c^4 (eq_single) is a quartic in e_x, b0 + b1 e_x
// + b2 e_x^2 + b3 e_x^3 + b4 e_x^4, with b0 = P(C0, S0), b1 = v dP/dc and
// b2, b3 from expanding it; b4 is the same for every row.  The pairs
// e_x = +-k share the even part b0 + b2 k^2 + b4 k^4 and the odd part
// k (b1 + b3 k^2): about 25 operations per row and 6 per pair.
struct RowQuartic {
    float v, v2, k3k6, k4k24, k6k24, a02x2, a21x2, b4;
};
__device__ __forceinline__ RowQuartic row_quartic_setup(const EqCoef &k, float v, float r2)
{
    RowQuartic q;
    q.v = v;
    q.v2 = v * v;
    q.k3k6 = 3.0f * k.k6;
    q.k4k24 = 4.0f * k.k24;
    q.k6k24 = 6.0f * k.k24;
    q.a02x2 = 2.0f * k.a02;
    q.a21x2 = 2.0f * k.a21;
    q.b4 = fmaf(k.a02, r2 * r2, fmaf(k.a21 * r2, q.v2, k.k24 * q.v2 * q.v2));
    return q;
}
// P at e_x = a - 3, a = 0..6, of the row with c = C0 + e_x v, s = S0 + r2 e_x^2.
__device__ __forceinline__ void row_quartic(const EqCoef &k, const RowQuartic &q, float r2, float C0, float S0,
                                            float (&P)[7])
{
    const float A0 = fmaf(S0, fmaf(S0, k.a02, k.a01), k.a00);
    const float A1 = fmaf(S0, k.a11, k.a10);
    const float A2 = fmaf(S0, k.a21, k.a20);
    const float b0 = fmaf(C0, fmaf(C0, fmaf(C0, fmaf(C0, k.k24, k.k6), A2), A1), A0);
    const float b1 = q.v * fmaf(C0, fmaf(C0, fmaf(C0, q.k4k24, q.k3k6), A2 + A2), A1);
    const float b2 = fmaf(r2, fmaf(C0, fmaf(C0, k.a21, k.a11), fmaf(q.a02x2, S0, k.a01)),
                          q.v2 * fmaf(C0, fmaf(C0, q.k6k24, q.k3k6), A2));
    const float b3 = q.v * fmaf(r2, fmaf(C0, q.a21x2, k.a11), q.v2 * fmaf(C0, q.k4k24, k.k6));
    P[3] = b0;
#pragma unroll
    for (int m = 1; m <= 3; ++m) {
        const float E = fmaf(q.b4, (float)(m * m * m * m), fmaf(b2, (float)(m * m), b0));
        const float O = (float)m * fmaf(b3, (float)(m * m), b1);
        P[3 + m] = E + O;
        P[3 - m] = E - O;
    }
}

// Pass 2 of one node and the rotational update: moments, equilibrium, BGK,
// store (the rest and the unit velocities deferred).  Each q_i = w_i P_i with
// P from the row quartic and w_i = (w_a w_b) w_c (an immediate times the
// plane's factor); the correction sums run over the q_i that are stored.
// Float storage: 10.4 ms per step on a 256^3 blast (n = 0) against 10.6 with
// the weight table and a polynomial per population.  The values of the e_z
// planes c < NS come from the stash, the others are pulled again.
template <bool ROT, int NS, typename ST>
__device__ __forceinline__ void q343_collide(const Params<kQ343, ST> &p, const Q343Weights &qw, const Offsets &o,
                                             int z, const Q343Sums &s, const ST *stash)
{
    constexpr int D = 3;
    constexpr int C = (kQ343 - 1) / 2;  // rest velocity (171)
    const int plane = p.pitch * p.Y;
    float h[7], R2 = 0.f;
    if (ROT) {
#pragma unroll
        for (int j = 0; j < 7; ++j) h[j] = ld(p, kQ343 + j, o.self());
#pragma unroll
        for (int k = 1; k <= 3; ++k) R2 = fmaf((float)(k * k), h[3 + k] + h[3 - k], R2);
    }
    const Moments m = make_moments<D, ROT>(p, s.rho, s.jx, s.jy, s.jz, s.e2, R2);
    if (!(m.rho > 0.f) || !(m.T > 0.f) || !(fabsf(m.T) < 3.0e38f)) atomicOr(p.status, 1);

    const float u2 = m.ux * m.ux + m.uy * m.uy + m.uz * m.uz;
    const float om_rho = p.omega * m.rho;
    const EqCoef k = eq_coef<D>(m.T, u2, om_rho);  // omega rho g^eq / w_i
    const float keep = 1.0f - p.omega;
    const float rux = m.ux * p.r, ruy = m.uy * p.r, ruz = m.uz * p.r;
    const int self = o.self();
    const RowQuartic rq = row_quartic_setup(k, rux, p.r2);
    float acc0 = 0.f, acc2 = 0.f, ax = 0.f, ay = 0.f, az = 0.f;
    float q_c = 0.f, q_mx = 0.f, q_px = 0.f, q_my = 0.f, q_py = 0.f, q_mz = 0.f, q_pz = 0.f;
    float g_c = 0.f, g_mx = 0.f, g_px = 0.f, g_my = 0.f, g_py = 0.f, g_mz = 0.f, g_pz = 0.f;
    // The correction sums are accumulated per row of 7 and then per plane, so
    // each carries the rounding of ~2 x 7 additions rather than of 343.
    // Planes in reverse order (see above).
    auto plane2 = [&](auto kept, int c) {
        constexpr bool KEPT = decltype(kept)::value;
        const int zo = bc_wrap(z - (c - 3), p.Z, p.bc2) * plane;
        const int ez = c - 3;
        const float wc = qw.wc[c];
        float p0 = 0.f, p2 = 0.f, px = 0.f, py = 0.f;  // plane sums
#pragma unroll
        for (int b = 0; b < 7; ++b) {
            const int row = zo + o.y[6 - b];
            const int ey = b - 3;
            const float cyz = fmaf((float)ey, ruy, (float)ez * ruz);
            const int e2yz_i = ey * ey + ez * ez;
            const float eyz2 = (float)e2yz_i;
            float Prow[7];
            row_quartic(k, rq, p.r2, cyz, p.r2 * eyz2, Prow);
            float r0 = 0.f, r2 = 0.f, rx = 0.f;  // row sums
#pragma unroll
            for (int a = 0; a < 7; ++a) {
                const int ex = a - 3;
                const int i = (c * 7 + b) * 7 + a;
                const int E2 = ex * ex + e2yz_i;
                const float q = (qw.w2[b * 7 + a] * wc) * Prow[a];  // w_i = (w_a w_b) w_c
                r0 += q;
                if (ex) {
                    r2 = fmaf((float)(ex * ex), q, r2);
                    rx = fmaf((float)ex, q, rx);
                }
                float g;
                if constexpr (KEPT) g = decode_pop(p, i, stash[i * kQ343Block + threadIdx.x]);
                else g = decode_pop(p, i, q343_load(p, i, row + o.x[6 - a]));
                if (E2 <= 1) {  // the rest and the six unit velocities: stored last
                    if (E2 == 0) { q_c = q; g_c = g; }
                    else if (ex == -1) { q_mx = q; g_mx = g; }
                    else if (ex == 1) { q_px = q; g_px = g; }
                    else if (ey == -1) { q_my = q; g_my = g; }
                    else if (ey == 1) { q_py = q; g_py = g; }
                    else if (ez == -1) { q_mz = q; g_mz = g; }
                    else { q_pz = q; g_pz = g; }
                } else {
                    q343_store(p, i, self, fmaf(keep, g, q));
                }
            }
            p0 += r0;
            p2 += fmaf(eyz2, r0, r2);
            px += rx;
            py = fmaf((float)ey, r0, py);
        }
        acc0 += p0;
        acc2 += p2;
        ax += px;
        ay += py;
        az = fmaf((float)ez, p0, az);
    };
    for (int c = 6; c >= 0; --c) {
        if (c < NS) plane2(std::true_type{}, c);
        else plane2(std::false_type{}, c);
    }
    const float d0 = om_rho - acc0;
    const float d2 = p.omega * m.E2_eq - acc2;
    const float bb = d2 * (0.5f / (float)D);
    const float dmx = 0.5f * (p.omega * m.j[0] - ax);
    const float dmy = 0.5f * (p.omega * m.j[1] - ay);
    const float dmz = 0.5f * (p.omega * m.j[2] - az);
    q343_store(p, C, self, fmaf(keep, g_c, q_c + (d0 - d2)));
    q343_store(p, C - 1, self, fmaf(keep, g_mx, q_mx + (bb - dmx)));
    q343_store(p, C + 1, self, fmaf(keep, g_px, q_px + (bb + dmx)));
    q343_store(p, C - 7, self, fmaf(keep, g_my, q_my + (bb - dmy)));
    q343_store(p, C + 7, self, fmaf(keep, g_py, q_py + (bb + dmy)));
    q343_store(p, C - 49, self, fmaf(keep, g_mz, q_mz + (bb - dmz)));
    q343_store(p, C + 49, self, fmaf(keep, g_pz, q_pz + (bb + dmz)));

    if (ROT) {
        float adv[7];
        rot_advect<D>(p, o, h, m, adv);
        rot_store(p, self, h, m, adv);
    }
}

// Pass 2 for 16-bit deviation storage (the factored-weight form above).
// Same structure as q343_collide: row and plane sums of w_i P_i, w_i |e_i|^2
// P_i and w_i e_i P_i, which are the sums of the post-collision equilibrium
// part q_i = w_i P_i, and the float32 corrections put on the rest and unit
// velocities (divided by their weights, since those are stored as
// deviations).
template <bool ROT, int NS, typename ST>
__device__ __forceinline__ void q343_collide_dev(const Params<kQ343, ST> &p, const Q343Weights &qw, const Offsets &o,
                                                 int z, const Q343Sums &s, const ST *stash)
{
    constexpr int D = 3;
    constexpr int C = (kQ343 - 1) / 2;  // rest velocity (171)
    const int plane = p.pitch * p.Y;
    float h[7], R2 = 0.f;
    if (ROT) {
#pragma unroll
        for (int j = 0; j < 7; ++j) h[j] = ld(p, kQ343 + j, o.self());
#pragma unroll
        for (int k = 1; k <= 3; ++k) R2 = fmaf((float)(k * k), h[3 + k] + h[3 - k], R2);
    }
    const Moments m = make_moments<D, ROT>(p, s.rho, s.jx, s.jy, s.jz, s.e2, R2);
    if (!(m.rho > 0.f) || !(m.T > 0.f) || !(fabsf(m.T) < 3.0e38f)) atomicOr(p.status, 1);

    const float u2 = m.ux * m.ux + m.uy * m.uy + m.uz * m.uz;
    const float om_rho = p.omega * m.rho;
    const EqCoef k = eq_coef<D>(m.T, u2, om_rho);  // P_i = omega rho g^eq_i / w_i
    const float keep = 1.0f - p.omega;
    const float rux = m.ux * p.r, ruy = m.uy * p.r, ruz = m.uz * p.r;
    const int self = o.self();
    float acc0 = 0.f, acc2 = 0.f, ax = 0.f, ay = 0.f, az = 0.f;
    float P_c = 0.f, P_mx = 0.f, P_px = 0.f, P_my = 0.f, P_py = 0.f, P_mz = 0.f, P_pz = 0.f;
    const RowQuartic rq = row_quartic_setup(k, rux, p.r2);
    float d_c = 0.f, d_mx = 0.f, d_px = 0.f, d_my = 0.f, d_py = 0.f, d_mz = 0.f, d_pz = 0.f;
    auto plane2 = [&](auto kept, int c) {
        constexpr bool KEPT = decltype(kept)::value;
        const int zo = bc_wrap(z - (c - 3), p.Z, p.bc2) * plane;
        const int ez = c - 3;
        const float ez2 = (float)(ez * ez);
        float p0 = 0.f, p2 = 0.f, px = 0.f, py = 0.f;  // plane sums (without w_c)
#pragma unroll
        for (int b = 0; b < 7; ++b) {
            const int row = zo + o.y[6 - b];
            const int ey = b - 3;
            const float cyz = fmaf((float)ey, ruy, (float)ez * ruz);
            const float eyz2 = (float)(ey * ey) + ez2;
            const float syz = p.r2 * eyz2;
            float Prow[7];
            row_quartic(k, rq, p.r2, cyz, syz, Prow);
            float r0 = 0.f, r2 = 0.f, rx = 0.f;  // row sums (without w_c)
#pragma unroll
            for (int a = 0; a < 7; ++a) {
                const int ex = a - 3;
                const int i = (c * 7 + b) * 7 + a;
                const float P = Prow[a];
                r0 = fmaf(qw.w2[b * 7 + a], P, r0);
                if (ex) {
                    r2 = fmaf(qw.w2x2[b * 7 + a], P, r2);
                    rx = fmaf(qw.w2x[b * 7 + a], P, rx);
                }
                float d;
                if constexpr (KEPT) d = Storage<ST>::to_dev(stash[i * kQ343Block + threadIdx.x]);
                else d = Storage<ST>::to_dev(q343_load(p, i, row + o.x[6 - a]));
                if (ex * ex + ey * ey + ez * ez <= 1) {  // the rest and the six unit velocities: stored last
                    if (ex == 0 && ey == 0 && ez == 0) { P_c = P; d_c = d; }
                    else if (ex == -1) { P_mx = P; d_mx = d; }
                    else if (ex == 1) { P_px = P; d_px = d; }
                    else if (ey == -1) { P_my = P; d_my = d; }
                    else if (ey == 1) { P_py = P; d_py = d; }
                    else if (ez == -1) { P_mz = P; d_mz = d; }
                    else { P_pz = P; d_pz = d; }
                } else {
                    q343_store_dev(p, i, self, fmaf(keep, d, P - p.omega));
                }
            }
            p0 += r0;
            p2 += fmaf(eyz2, r0, r2);
            px += rx;
            py = fmaf((float)ey, r0, py);
        }
        const float wc = qw.wc[c];
        acc0 = fmaf(wc, p0, acc0);
        acc2 = fmaf(wc, p2, acc2);
        ax = fmaf(wc, px, ax);
        ay = fmaf(wc, py, ay);
        az = fmaf(wc * (float)ez, p0, az);
    };
    for (int c = 6; c >= 0; --c) {
        if (c < NS) plane2(std::true_type{}, c);
        else plane2(std::false_type{}, c);
    }
    const float d0 = om_rho - acc0;
    const float d2 = p.omega * m.E2_eq - acc2;
    const float bb = d2 * (0.5f / (float)D);
    const float dmx = 0.5f * (p.omega * m.j[0] - ax);
    const float dmy = 0.5f * (p.omega * m.j[1] - ay);
    const float dmz = 0.5f * (p.omega * m.j[2] - az);
    const float iw0 = qw.iw_rest, iw1 = qw.iw_unit;
    q343_store_dev(p, C, self, fmaf(keep, d_c, fmaf(d0 - d2, iw0, P_c - p.omega)));
    q343_store_dev(p, C - 1, self, fmaf(keep, d_mx, fmaf(bb - dmx, iw1, P_mx - p.omega)));
    q343_store_dev(p, C + 1, self, fmaf(keep, d_px, fmaf(bb + dmx, iw1, P_px - p.omega)));
    q343_store_dev(p, C - 7, self, fmaf(keep, d_my, fmaf(bb - dmy, iw1, P_my - p.omega)));
    q343_store_dev(p, C + 7, self, fmaf(keep, d_py, fmaf(bb + dmy, iw1, P_py - p.omega)));
    q343_store_dev(p, C - 49, self, fmaf(keep, d_mz, fmaf(bb - dmz, iw1, P_mz - p.omega)));
    q343_store_dev(p, C + 49, self, fmaf(keep, d_pz, fmaf(bb + dmz, iw1, P_pz - p.omega)));

    if (ROT) {
        float adv[7];
        rot_advect<D>(p, o, h, m, adv);
        rot_store(p, self, h, m, adv);
    }
}

// One launch: pass 1, then pass 2 on the same thread.
template <bool ROT, typename ST>
__global__ void __launch_bounds__(kQ343Block, LBM_Q343_MIN_BLOCKS)
    k_step_q343(const Params<kQ343, ST> p, const Q343Weights qw)
{
    const int x = blockIdx.x * kQ343Block + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= p.X) return;
    const Offsets o = node_offsets<3>(p, x, y, z);
    extern __shared__ unsigned char q343_smem[];
    ST *stash = reinterpret_cast<ST *>(q343_smem);  // [NS planes x 49][kQ343Block] raw values
    constexpr int NS = StashPlanes<ST>::value;
    const Q343Sums s = q343_sums<NS>(p, o, z, stash);
    if constexpr (Q343Dev<ST>::value) q343_collide_dev<ROT, NS>(p, qw, o, z, s, stash);
    else q343_collide<ROT, NS>(p, qw, o, z, s, stash);
}

}  // namespace

template <bool ROT, typename ST> cudaError_t launch_step_q343(const Args &a, cudaStream_t s)
{
    const auto p = make_params<kQ343, ST>(a);
    const dim3 grid((a.X + kQ343Block - 1) / kQ343Block, a.Y, a.Z);
    constexpr size_t sh = stash_bytes<ST>();
    if constexpr (sh > 48 * 1024) {  // the opt-in limit is a per-device function attribute
        static std::atomic<bool> done[64];
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
        if (!done[dev].load()) {
            e = cudaFuncSetAttribute(k_step_q343<ROT, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sh);
            if (e != cudaSuccess) return e;
            done[dev].store(true);
        }
    }
    Q343Weights qw;
    for (int b = 0; b < 7; ++b)
        for (int c = 0; c < 7; ++c) {
            const double wab = (double)a.wr[c] * (double)a.wr[b];
            qw.w2[b * 7 + c] = (float)wab;
            qw.w2x[b * 7 + c] = (float)(wab * (c - 3));
            qw.w2x2[b * 7 + c] = (float)(wab * (c - 3) * (c - 3));
        }
    for (int c = 0; c < 7; ++c) qw.wc[c] = a.wr[c];
    qw.iw_rest = (float)(1.0 / ((double)a.wr[3] * (double)a.wr[3] * (double)a.wr[3]));
    qw.iw_unit = (float)(1.0 / ((double)a.wr[2] * (double)a.wr[3] * (double)a.wr[3]));
    k_step_q343<ROT, ST><<<grid, kQ343Block, sh, s>>>(p, qw);
    return cudaGetLastError();
}

cudaError_t launch_d3q343(Op op, const Args &a, cudaStream_t s) { return launch_lattice<4>(op, a, s); }

}  // namespace lbm
