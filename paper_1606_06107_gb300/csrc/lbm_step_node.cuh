// The STREAM step for per-node reference storage (LBM_STORE_F16_NODE /
// LBM_STORE_BF16_NODE) on the 1-D and 2-D lattices.  Included by
// lbm_step.cuh inside namespace lbm; uses its lattices, parameters,
// equilibria, moments and reference records (ref_dev).
//
// Stored format: a translational value is s_i = f_i / w_i - R_i with R_i the
// node's reference (Params: first order in u, up to second order in T - 1 of
// the Hermite equilibrium), a rotational value s_j = h_j / w_j - h_j^eq(T) / w_j,
// in IEEE half or bfloat16; each node's record (rho - 1, rho t / 2, rho r u_x,
// rho r u_y) follows the populations.  All arithmetic is float32, except the
// temperature's kinetic-energy subtraction, which is double (make_moments).
//
// The kernel computes on the deviations from rest d = f / w - 1: the pull
// adds the reference deviation ref_dev() of the source node's record to the
// stored value, the post-collision deviation is
// d* = (1 - omega) d + omega rho P - omega (P = g^eq / (w rho)), so a value
// needs no multiply-add to decode or encode, and the moment sums are
// sum_i w_i d_i plus the constant lattice sums of the float weights.  The
// store subtracts the reference deviation of the node's new record, the
// moments just taken, which it also writes.  The rotational update works on
// deviations too (the upwind stencil of a constant is zero); each value of
// its stencil is decoded with the record of the node it is read from.
//
// Measured and dropped: the same deviation-space form for rest storage
// (68.3 warp instructions per node against 63.6 for k_step with 16-bit
// values, 2 % slower); two x-adjacent nodes per thread with packed 32-bit
// loads and stores (17 % fewer instructions per node but 168 registers, so
// 11 resident warps per SM instead of 19, 30 % slower); one pointer per
// source column with block-uniform row offsets (5 % more instructions than
// integer offsets); the block's 7 x 134 source records staged in shared
// memory once instead of each value loading its record from L1 (6.8 against
// 7.8 Gnode/s: the barrier and the staging cost more than the L1 hits).
#pragma once

// Resident 128-thread blocks per SM the register allocation must allow
// (A/B on the 2048^2 workload: 3 / 4 / 5 / 6 blocks gave 6,969 / 8,089 /
// 8,187 / 7,870 Mnode/s with bfloat16 node references).
#ifndef LBM_STEP_NODE_MIN_BLOCKS
#define LBM_STEP_NODE_MIN_BLOCKS 5
#endif

template <typename ST> struct Dev16;
template <> struct Dev16<__half> {
    __device__ static float get(unsigned short v) { return __half2float(__ushort_as_half(v)); }
    __device__ static unsigned short put(float f) { return __half_as_ushort(__float2half_rn(f)); }
};
template <> struct Dev16<__nv_bfloat16> {
    __device__ static float get(unsigned short v) { return __uint_as_float((uint32_t)v << 16); }
    __device__ static unsigned short put(float f) { return __bfloat16_as_ushort(__float2bfloat16_rn(f)); }
};

template <int LAT, bool ROT, typename ST>
__global__ void __launch_bounds__(kBlockX, LBM_STEP_NODE_MIN_BLOCKS)
k_step_node(const Params<Lattice<LAT>::Q, ST> p)
{
    using L = Lattice<LAT>;
    using DV = Dev16<typename NodeRef<ST>::elem>;
    constexpr int Q = L::Q;
    constexpr int D = L::D;
    constexpr int C = (Q - 1) / 2;
    static_assert(D <= 2, "D3Q343 has its own kernel");
    const int x = blockIdx.x * kBlockX + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= p.X) return;
    const unsigned short *src = reinterpret_cast<const unsigned short *>(p.src);
    unsigned short *dst = reinterpret_cast<unsigned short *>(p.dst);
    // source columns x - 3 .. x + 3 and rows y - 3 .. y + 3, wrapped or clamped
    int ox[7], oy[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        ox[k] = bc_wrap(x + k - 3, p.X, p.bc0);
        oy[k] = (D >= 2) ? bc_wrap(y + k - 3, p.Y, p.bc1) * p.pitch : 0;
    }
    const uint32_t S = (uint32_t)p.S;
    const int self = oy[3] + ox[3];

    // ---- pull the deviations: g_i(x) = ft_i(x - e_i) ----------------------
    float d[Q], h[7];
    static_for<0, Q>([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        constexpr int ex = L::ex(I), ey = L::ey(I);
        const int off = oy[3 - ey] + ox[3 - ex];
        d[I] = DV::get(__ldg(src + ((uint32_t)I * S + (uint32_t)off)));
        d[I] += ref_dev(p, I, __ldg(p.ref_src + off), (float)ex, (float)ey, p.kmD[I], p.kt2[I]);
    });
    float t_self = 0.f;
    if (ROT) {
        t_self = ref_t(__ldg(p.ref_src + self));
#pragma unroll
        for (int j = 0; j < 7; ++j) {
            h[j] = DV::get(__ldg(src + ((uint32_t)(Q + j) * S + (uint32_t)self)));
            h[j] += t_self * fmaf(t_self, p.hb[j], p.ha[j]);
        }
    }

    // ---- moments: partial sums of w_i d_i by column and row ---------------
    Moments m;
    {
        float cs[7], rs[7];
        bool hc[7] = {}, hr[7] = {};
#pragma unroll
        for (int k = 0; k < 7; ++k) cs[k] = rs[k] = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int a = L::ex(i) + 3, b = L::ey(i) + 3;
            cs[a] = hc[a] ? fmaf(p.w[i], d[i], cs[a]) : p.w[i] * d[i];
            hc[a] = true;
            if (D >= 2) { rs[b] = hr[b] ? fmaf(p.w[i], d[i], rs[b]) : p.w[i] * d[i]; hr[b] = true; }
        }
        float rho = cs[3], jx = 0.f, jy = 0.f, e2 = 0.f;
#pragma unroll
        for (int k = 1; k <= 3; ++k) {
            const float s = (float)k, ss = (float)(k * k);
            rho += cs[3 + k] + cs[3 - k];
            jx = fmaf(s, cs[3 + k] - cs[3 - k], jx);
            e2 = fmaf(ss, cs[3 + k] + cs[3 - k], e2);
            if (D >= 2) {
                jy = fmaf(s, rs[3 + k] - rs[3 - k], jy);
                e2 = fmaf(ss, rs[3 + k] + rs[3 - k], e2);
            }
        }
        float R2 = 0.f;
        if (ROT) {
#pragma unroll
            for (int k = 1; k <= 3; ++k)
                R2 = fmaf((float)(k * k), fmaf(p.wr[3 + k], h[3 + k], p.wr[3 - k] * h[3 - k]), R2);
            R2 += p.swr2;
        }
        m = make_moments<D, ROT>(p, rho + p.sw0, jx, jy, 0.f, e2 + p.sw2, R2);
    }
    if (!(m.rho > 0.f) || !(m.T > 0.f) || !(fabsf(m.T) < 3.0e38f)) atomicOr(p.status, 1);

    // ---- collision in deviation space, stores -----------------------------
    unsigned short *out = dst + self;
    const float om = p.omega, keep = 1.0f - p.omega;
    const EqCoef k = eq_coef<D>(m.T, m.ux * m.ux + m.uy * m.uy, p.omega * m.rho);  // omega rho P
    const float ru[2] = {m.ux * p.r, m.uy * p.r};
    // this node's new reference record (what the next step's readers decode with)
    const float4 rc = make_float4(m.rho - 1.0f, 0.5f * (m.rho * (m.T - 1.0f)), m.rho * ru[0], m.rho * ru[1]);
    p.ref_dst[self] = rc;
    auto put = [&](int pop, float ex, float ey, float kmd, float v) {
        v -= ref_dev(p, pop, rc, ex, ey, kmd, p.kt2[pop]);
        out[(uint32_t)pop * S] = DV::put(v);
    };
    float acc0 = 0.f, acc2 = 0.f, accj[2] = {0.f, 0.f}, qm[2] = {0.f, 0.f}, qp[2] = {0.f, 0.f};
    static_for<0, C>([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        constexpr int J = Q - 1 - I;
        constexpr int E2 = e2_of<LAT>(I);
        constexpr int e[2] = {L::ex(I), L::ey(I)};
        float c = 0.f;
#pragma unroll
        for (int a = 0; a < D; ++a)
            if (e[a]) c = fmaf((float)e[a], ru[a], c);
        float Pp, Pm;
        eq_pair(k, c, p.r2 * (float)E2, Pp, Pm);
        const float sum = Pp + Pm, diff = Pp - Pm;
        acc0 = fmaf(p.w[I], sum, acc0);  // w(-e) = w(e)
        acc2 = fmaf(p.w[I] * (float)E2, sum, acc2);
#pragma unroll
        for (int a = 0; a < D; ++a)
            if (e[a]) accj[a] = fmaf(p.w[I] * (float)e[a], diff, accj[a]);
        if constexpr (E2 == 1) {  // I is -1_a: stored last, corrected
            constexpr int ax = e[0] ? 0 : 1;
            qm[ax] = Pp;
            qp[ax] = Pm;
        } else {
            put(I, (float)e[0], (float)e[1], p.kmD[I], fmaf(keep, d[I], Pp - om));
            put(J, (float)-e[0], (float)-e[1], p.kmD[J], fmaf(keep, d[J], Pm - om));
        }
    });
    // rest and unit velocities with the float32 moment corrections of
    // collide_store, each defect divided by the weight of its carrier
    const float q_c = k.a00;
    acc0 = fmaf(p.w[C], q_c, acc0);
    const float d0 = p.omega * m.rho - acc0;
    const float d2 = p.omega * m.E2_eq - acc2;
    const float b = d2 * (0.5f / (float)D);
    put(C, 0.f, 0.f, p.kmD[C], fmaf(keep, d[C], (q_c - om) + (d0 - d2) * p.iw[C]));
    static_for<0, D>([&](auto ac) {
        constexpr int A = decltype(ac)::value;
        constexpr int IM = index_of<LAT>(A == 0 ? -1 : 0, A == 1 ? -1 : 0, 0);
        constexpr int IP = Q - 1 - IM;
        const float dm = 0.5f * (p.omega * m.j[A] - accj[A]);
        const float sx = (A == 0) ? 1.f : 0.f, sy = (A == 1) ? 1.f : 0.f;
        put(IM, -sx, -sy, p.kmD[IM], fmaf(keep, d[IM], (qm[A] - om) + (b - dm) * p.iw[IM]));
        put(IP, sx, sy, p.kmD[IP], fmaf(keep, d[IP], (qp[A] - om) + (b + dm) * p.iw[IP]));
    });

    // ---- rotational populations: upwind advection of the deviations -------
    if (ROT) {
        float heq[7], adv[7], adv_t1 = 0.f, adv_t2 = 0.f;
        const float t_new = ref_t(rc);
        heq_node(p, m.T, m.T_lat, heq);
#pragma unroll
        for (int j = 0; j < 7; ++j) adv[j] = 0.f;
        // One axis: the values two and one nodes upwind and one downwind.
        // Each neighbour value adds t (ha_j + t hb_j) of its own
        // node, so their references enter as ha_j T1 + hb_j T2, with T1, T2
        // the stencil applied to t and t^2 of the three neighbours (this
        // node's own value h[j] is decoded already, its stencil slot is 0).
        auto axis = [&](float nu, int uu, int u1, int d1) {
            const float anu = fabsf(nu);
#pragma unroll
            for (int j = 0; j < 7; ++j) {
                const uint32_t o = (uint32_t)(Q + j) * S;
                adv[j] += upwind_abs(anu, DV::get(__ldg(src + (o + (uint32_t)uu))),
                                     DV::get(__ldg(src + (o + (uint32_t)u1))), h[j],
                                     DV::get(__ldg(src + (o + (uint32_t)d1))));
            }
            const float tuu = ref_t(__ldg(p.ref_src + uu)), tu1 = ref_t(__ldg(p.ref_src + u1));
            const float td1 = ref_t(__ldg(p.ref_src + d1));
            adv_t1 += upwind_abs(anu, tuu, tu1, 0.f, td1);
            adv_t2 += upwind_abs(anu, tuu * tuu, tu1 * tu1, 0.f, td1 * td1);
        };
        {
            const float nu = m.ux * p.nu_scale;
            const bool pos = nu >= 0.0f;
            axis(nu, oy[3] + (pos ? ox[1] : ox[5]), oy[3] + (pos ? ox[2] : ox[4]), oy[3] + (pos ? ox[4] : ox[2]));
        }
        if (D >= 2) {
            const float nu = m.uy * p.nu_scale;
            const bool pos = nu >= 0.0f;
            axis(nu, (pos ? oy[1] : oy[5]) + ox[3], (pos ? oy[2] : oy[4]) + ox[3], (pos ? oy[4] : oy[2]) + ox[3]);
        }
        // d* = (1 - omega) d + omega (h^eq / w - 1) - advection of d
#pragma unroll
        for (int j = 0; j < 7; ++j) {
            float a = adv[j];
            a = fmaf(p.ha[j], adv_t1, fmaf(p.hb[j], adv_t2, a));
            float v = fmaf(keep, h[j], fmaf(om, heq[j] * p.iwr[j], -om) - a);
            v -= t_new * fmaf(t_new, p.hb[j], p.ha[j]);
            out[(uint32_t)(Q + j) * S] = DV::put(v);
        }
    }
}
