// Host side of the C ABI declared in include/lbm.h: argument validation, the
// lattice constants (solved here in double precision, independently of any
// other component), buffer binding and kernel launches.  The library never
// allocates device memory: every device buffer belongs to the caller.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include <cuda_runtime.h>

#include "../../include/lbm.h"
#include "lbm_internal.h"

using lbm::Args;
using lbm::Op;

struct lbm_ctx {
    int D = 0, lattice = 0, n = 0, Q = 0, Qr = 0;
    int mode = LBM_MODE_STREAM, m_fd = 1;
    int storage = LBM_STORE_F32;
    double tau = 0.0;
    double r = 0.0;
    double w[lbm::kMaxQ] = {};
    int e[lbm::kMaxQ][3] = {};
    double wr[7] = {};
    int64_t shape[3] = {1, 1, 1};
    int bc[3] = {0, 0, 0};
    int pitch = 0;
    int64_t S = 0, N = 0;
    size_t state_bytes = 0, work_bytes = 0, ref_offset = 0;
    bool grid_set = false, bound = false, has_state = false;
    void *buf[2] = {nullptr, nullptr};
    int cur = 0;
    char *work = nullptr;
    cudaStream_t stream = nullptr;
    int device = 0;
    int red_blocks = 1;    int64_t steps = 0;
    int64_t launches = 0;
    std::string err;
};

namespace {

int fail(lbm_ctx *h, int code, const std::string &msg)
{
    if (h) h->err = msg;
    return code;
}

int cuda_fail(lbm_ctx *h, cudaError_t e, const char *where)
{
    return fail(h, LBM_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Makes the handle's device current for the duration of one API call.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// ---------------------------------------------------------------------------
// Lattice constants.  The scaling factor r and the weights of Tables I and II
// are the Gauss-Hermite quadratures that reproduce the moments of the unit
// normal distribution.  Here, for a trial r, the weights follow from a linear
// subset of the moment equations; r is then the root of the one remaining
// equation, found by bisection.

double dfact(int k)  // (k-1)!! for even k >= 0: E[x^k] of N(0,1)
{
    double m = 1.0;
    for (int j = k - 1; j > 1; j -= 2) m *= j;
    return m;
}

bool solve_linear(int n, double *A, double *b)
{
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[r * n + c]) > std::fabs(A[p * n + c])) p = r;
        if (A[p * n + c] == 0.0) return false;
        for (int k = 0; k < n; ++k) std::swap(A[c * n + k], A[p * n + k]);
        std::swap(b[c], b[p]);
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double f = A[r * n + c] / A[c * n + c];
            for (int k = 0; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
            b[r] -= f * b[c];
        }
    }
    for (int c = 0; c < n; ++c) b[c] /= A[c * n + c];
    return true;
}

// D1Q7: velocities 0, +-r, +-2r, +-3r with weights v[0..3].  Moments 2, 4, 6
// fix v[1..3]; mass fixes v[0]; returns the residual of the 8th moment.
double d1q7_for_r(double r, double v[4])
{
    double A[9], b[3];
    for (int k = 0; k < 3; ++k) {
        const int p = 2 * (k + 1);
        for (int m = 1; m <= 3; ++m) A[k * 3 + (m - 1)] = 2.0 * std::pow(m * r, p);
        b[k] = dfact(p);
    }
    solve_linear(3, A, b);
    v[1] = b[0]; v[2] = b[1]; v[3] = b[2];
    v[0] = 1.0 - 2.0 * (v[1] + v[2] + v[3]);
    double m8 = 0.0;
    for (int m = 1; m <= 3; ++m) m8 += 2.0 * v[m] * std::pow(m * r, 8);
    return m8 - dfact(8);
}

bool d2q37_member(int ex, int ey)
{
    const int a = std::abs(ex), b = std::abs(ey);
    return !((a == 2 && b == 2) || (a == 2 && b == 3) || (a == 3 && b == 2));
}

// symmetry group of a D2Q37 velocity: (0,0) (1,0) (1,1) (2,0) (2,1) (3,0) (3,1) (3,3)
int d2q37_group(int ex, int ey)
{
    const int a = std::max(std::abs(ex), std::abs(ey)), b = std::min(std::abs(ex), std::abs(ey));
    static const int base[8][2] = {{0, 0}, {1, 0}, {1, 1}, {2, 0}, {2, 1}, {3, 0}, {3, 1}, {3, 3}};
    for (int g = 0; g < 8; ++g)
        if (base[g][0] == a && base[g][1] == b) return g;
    return -1;
}

// D2Q37: group weights W[1..7] from the moments x^2, x^4, x^2y^2, x^6, x^4y^2,
// x^6y^2, x^4y^4; W[0] from mass; returns the residual of the x^8 moment.
double d2q37_for_r(double r, double W[8])
{
    static const int eq[7][2] = {{2, 0}, {4, 0}, {2, 2}, {6, 0}, {4, 2}, {6, 2}, {4, 4}};
    double A[49] = {}, b[7], S8[8] = {}, cnt[8] = {};
    for (int ey = -3; ey <= 3; ++ey)
        for (int ex = -3; ex <= 3; ++ex) {
            if (!d2q37_member(ex, ey)) continue;
            const int g = d2q37_group(ex, ey);
            cnt[g] += 1.0;
            S8[g] += std::pow(r * ex, 8);
            if (g == 0) continue;
            for (int q = 0; q < 7; ++q)
                A[q * 7 + (g - 1)] += std::pow(r * ex, eq[q][0]) * std::pow(r * ey, eq[q][1]);
        }
    for (int q = 0; q < 7; ++q) b[q] = dfact(eq[q][0]) * dfact(eq[q][1]);
    solve_linear(7, A, b);
    double mass = 0.0, m8 = 0.0;
    for (int g = 1; g < 8; ++g) {
        W[g] = b[g - 1];
        mass += cnt[g] * W[g];
        m8 += W[g] * S8[g];
    }
    W[0] = 1.0 - mass;
    return m8 - dfact(8);
}

template <typename F> double bisect_r(F resid)
{
    double lo = 1.15, hi = 1.25;
    double flo = resid(lo);
    for (int it = 0; it < 200 && hi - lo > 1e-16; ++it) {
        const double mid = 0.5 * (lo + hi);
        const double fm = resid(mid);
        if ((fm < 0) == (flo < 0)) { lo = mid; flo = fm; }
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

// Fills r, e (canonical (ez,ey,ex) order) and w; returns Q or -1.
int lattice_constants(int lattice, double *r, int e[][3], double *w)
{
    double v[4];
    const double r1 = bisect_r([&](double x) { return d1q7_for_r(x, v); });
    d1q7_for_r(r1, v);
    if (lattice == LBM_D1Q7) {
        *r = r1;
        for (int i = 0; i < 7; ++i) {
            e[i][0] = i - 3; e[i][1] = 0; e[i][2] = 0;
            w[i] = v[std::abs(i - 3)];
        }
        return 7;
    }
    if (lattice == LBM_D2Q49) {
        *r = r1;
        for (int i = 0; i < 49; ++i) {
            const int ex = i % 7 - 3, ey = i / 7 - 3;
            e[i][0] = ex; e[i][1] = ey; e[i][2] = 0;
            w[i] = v[std::abs(ex)] * v[std::abs(ey)];
        }
        return 49;
    }
    if (lattice == LBM_D3Q343) {
        *r = r1;
        for (int i = 0; i < 343; ++i) {
            const int ex = i % 7 - 3, ey = (i / 7) % 7 - 3, ez = i / 49 - 3;
            e[i][0] = ex; e[i][1] = ey; e[i][2] = ez;
            w[i] = v[std::abs(ex)] * v[std::abs(ey)] * v[std::abs(ez)];
        }
        return 343;
    }
    if (lattice == LBM_D2Q37) {
        double W[8];
        *r = bisect_r([&](double x) { return d2q37_for_r(x, W); });
        d2q37_for_r(*r, W);
        int q = 0;
        for (int ey = -3; ey <= 3; ++ey)
            for (int ex = -3; ex <= 3; ++ex) {
                if (!d2q37_member(ex, ey)) continue;
                e[q][0] = ex; e[q][1] = ey; e[q][2] = 0;
                w[q] = W[d2q37_group(ex, ey)];
                ++q;
            }
        return q;
    }
    return -1;
}

int lattice_dim(int lattice)
{
    switch (lattice) {
    case LBM_D1Q7: return 1;
    case LBM_D2Q37: case LBM_D2Q49: return 2;
    case LBM_D3Q343: return 3;
    default: return 0;
    }
}

// ---------------------------------------------------------------------------
// Launch plumbing.

Args make_args(const lbm_ctx *h)
{
    Args a{};
    a.lattice = h->lattice;
    a.D = h->D;
    a.Q = h->Q;
    a.Qr = h->Qr;
    a.mode = h->mode;
    a.m_fd = h->m_fd;
    a.storage = h->storage;
    a.ref_offset = h->ref_offset;
    a.X = (int)h->shape[0];
    a.Y = (int)h->shape[1];
    a.Z = (int)h->shape[2];
    a.pitch = h->pitch;
    a.S = h->S;
    a.N = h->N;
    for (int k = 0; k < 3; ++k) a.bc[k] = h->bc[k];
    const double m = (h->mode == LBM_MODE_FD) ? h->m_fd : 1.0;
    a.r = (float)h->r;
    // omega and 1 - omega must both be exact floats: the kernels keep
    // (1 - omega) g and add omega g^eq, and a rounded 1 - omega would create
    // or destroy mass at ~1e-8 per step.  Nudge omega by at most half an ulp.
    const float om = (float)(1.0 / (m * h->tau));
    const float keep = (float)(1.0 - (double)om);
    a.omega = (float)(1.0 - (double)keep);
    a.nu_scale = (float)(1.0 / (m * h->r));
    a.cT = (float)(0.5 * (h->D + h->n));  // T = (energy per mass) / ((D+n)/2), Eq. T
    a.half_n_r2 = (float)(0.5 * h->n * h->r * h->r);
    a.half_n = (float)(0.5 * h->n);
    a.inv_m = (float)(1.0 / m);
    for (int i = 0; i < h->Q; ++i) a.w[i] = (float)h->w[i];
    for (int j = 0; j < 7; ++j) a.wr[j] = (float)h->wr[j];
    a.status = reinterpret_cast<int *>(h->work + lbm::kWorkStatus);
    a.partials = reinterpret_cast<double *>(h->work + lbm::kWorkPartials);
    a.red_blocks = h->red_blocks;
    return a;
}

cudaError_t launch(lbm_ctx *h, Op op, const Args &a)
{
    ++h->launches;
    switch (h->lattice) {
    case LBM_D1Q7: return lbm::launch_d1q7(op, a, h->stream);
    case LBM_D2Q37: return lbm::launch_d2q37(op, a, h->stream);
    case LBM_D2Q49: return lbm::launch_d2q49(op, a, h->stream);
    case LBM_D3Q343: return lbm::launch_d3q343(op, a, h->stream);
    default: return cudaErrorInvalidValue;
    }
}

__global__ void k_finalize(const double *partials, int nblocks, double *result)
{
    using lbm::kRedSlots;
    double acc[kRedSlots] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int k = 0; k < kRedSlots; ++k) {
            const double v = partials[(size_t)b * kRedSlots + k];
            acc[k] = (k == 5) ? fmax(acc[k], v) : acc[k] + v;
        }
    __shared__ double red[kRedSlots][lbm::kRedThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < kRedSlots; ++k) {
        double v = acc[k];
        for (int off = 16; off > 0; off >>= 1) {
            const double o = __shfl_down_sync(0xffffffffu, v, off);
            v = (k == 5) ? fmax(v, o) : v + o;
        }
        if (lane == 0) red[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < kRedSlots) {
        const int k = threadIdx.x;
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) v = (k == 5) ? fmax(v, red[k][w]) : v + red[k][w];
        result[k] = v;
    }
}

bool aligned256(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 255u) == 0; }

}  // namespace

// ---------------------------------------------------------------------------
// C ABI

extern "C" {

int lbm_lattice_info(int lattice, double *r, int *e, double *w)
{
    if (!r || !e || !w) return LBM_EINVAL;
    double rr, ww[lbm::kMaxQ];
    int ee[lbm::kMaxQ][3];
    const int q = lattice_constants(lattice, &rr, ee, ww);
    if (q < 0) return LBM_EINVAL;
    *r = rr;
    for (int i = 0; i < q; ++i) {
        for (int a = 0; a < 3; ++a) e[i * 3 + a] = ee[i][a];
        w[i] = ww[i];
    }
    return q;
}

int lbm_create(int D, int lattice, int n, double tau, lbm_handle *out)
{
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    if (D < 1 || D > 3) return LBM_EINVAL;
    if (lattice_dim(lattice) != D) return LBM_EINVAL;
    if (n < 0 || !(tau > 0.0) || !std::isfinite(tau)) return LBM_EINVAL;
    lbm_ctx *h = new lbm_ctx();
    h->D = D;
    h->lattice = lattice;
    h->n = n;
    h->tau = tau;
    const int q = lattice_constants(lattice, &h->r, h->e, h->w);
    if (q < 0) {
        delete h;
        return LBM_EINVAL;
    }
    h->Q = q;
    h->Qr = n > 0 ? 7 : 0;
    double r1, w1[7];
    int e1[lbm::kMaxQ][3];
    lattice_constants(LBM_D1Q7, &r1, e1, w1);
    for (int j = 0; j < 7; ++j) h->wr[j] = w1[j];
    cudaGetDevice(&h->device);
    *out = h;
    return LBM_OK;
}

int lbm_set_storage(lbm_handle h, int storage)
{
    if (!h) return LBM_EINVAL;
    if (h->grid_set) return fail(h, LBM_ESTATE, "lbm_set_storage must precede lbm_set_grid");
    if (storage < LBM_STORE_F32 || storage > LBM_STORE_BF16_NODE)
        return fail(h, LBM_EINVAL, "unknown storage");
    h->storage = storage;
    return LBM_OK;
}

int lbm_set_mode(lbm_handle h, int mode, int m_fd)
{
    if (!h) return LBM_EINVAL;
    if (h->grid_set) return fail(h, LBM_ESTATE, "lbm_set_mode must precede lbm_set_grid");
    if (mode != LBM_MODE_STREAM && mode != LBM_MODE_FD) return fail(h, LBM_EINVAL, "unknown mode");
    if (mode == LBM_MODE_FD && m_fd < 1) return fail(h, LBM_EINVAL, "m_fd must be >= 1");
    if (mode == LBM_MODE_FD && h->lattice == LBM_D3Q343)
        return fail(h, LBM_EINVAL, "D3Q343 has STREAM transport only");
    h->mode = mode;
    h->m_fd = (mode == LBM_MODE_FD) ? m_fd : 1;
    return LBM_OK;
}

int lbm_set_grid(lbm_handle h, const int64_t *shape, const int *bc, size_t *state_bytes,
                 size_t *work_bytes)
{
    if (!h) return LBM_EINVAL;
    if (!shape || !bc) return fail(h, LBM_EINVAL, "shape and bc are required");
    if (h->bound) return fail(h, LBM_ESTATE, "grid already bound to buffers");
    int64_t s[3] = {1, 1, 1};
    int b[3] = {0, 0, 0};
    for (int a = 0; a < h->D; ++a) {
        if (shape[a] < 1) return fail(h, LBM_ESIZE, "every extent must be >= 1");
        if (bc[a] != LBM_BC_PERIODIC && bc[a] != LBM_BC_COPY) return fail(h, LBM_EINVAL, "unknown bc");
        s[a] = shape[a];
        b[a] = bc[a];
    }
    if (s[0] > (int64_t)1 << 30 || s[1] > 65535 || s[2] > 65535)
        return fail(h, LBM_ESIZE, "X <= 2^30 and Y, Z <= 65535 are required");
    const bool node_ref = h->storage == LBM_STORE_F16_NODE || h->storage == LBM_STORE_BF16_NODE;
    if (node_ref && (h->lattice == LBM_D3Q343 || h->mode != LBM_MODE_STREAM))
        return fail(h, LBM_EINVAL, "per-node reference storage needs STREAM mode and a 1-D or 2-D lattice");
    const size_t elem = (h->storage == LBM_STORE_F32) ? sizeof(float) : 2;
    const int64_t row_align = 128 / (int64_t)elem;  // rows start on 128-byte lines
    const int64_t pitch = (s[0] + row_align - 1) / row_align * row_align;
    const int64_t S = pitch * s[1] * s[2];
    // the kernels index the whole state buffer with 32-bit element offsets
    // the kernels index up to 49 populations with 32-bit element offsets
    // (D3Q343 uses 64-bit ones); every per-population offset is 32-bit
    if (S > 0x7fffffffLL || (h->Q <= 49 && S * (h->Q + h->Qr) > 0x7fffffffLL))
        return fail(h, LBM_ESIZE, "state buffer would exceed 2^31 floats");
    for (int a = 0; a < 3; ++a) {
        h->shape[a] = s[a];
        h->bc[a] = b[a];
    }
    h->pitch = (int)pitch;
    h->S = S;
    h->N = s[0] * s[1] * s[2];
    h->state_bytes = elem * (size_t)(h->Q + h->Qr) * (size_t)S;
    h->ref_offset = 0;
    if (node_ref) {  // the reference records follow the populations, 256-byte aligned
        h->ref_offset = (h->state_bytes + 255) / 256 * 256;
        h->state_bytes = h->ref_offset + 16 * (size_t)S;
    }
    h->work_bytes = lbm::kWorkBytes;
    h->grid_set = true;
    if (state_bytes) *state_bytes = h->state_bytes;
    if (work_bytes) *work_bytes = h->work_bytes;
    return LBM_OK;
}

int lbm_bind(lbm_handle h, void *buf_a, void *buf_b, size_t state_bytes, void *work,
             size_t work_bytes, void *stream)
{
    if (!h) return LBM_EINVAL;
    if (!h->grid_set) return fail(h, LBM_ESTATE, "lbm_set_grid must precede lbm_bind");
    if (!buf_a || !buf_b || !work) return fail(h, LBM_EINVAL, "null buffer");
    if (buf_a == buf_b) return fail(h, LBM_EINVAL, "the two state buffers must differ");
    if (!aligned256(buf_a) || !aligned256(buf_b) || !aligned256(work))
        return fail(h, LBM_EINVAL, "buffers must be 256-byte aligned");
    if (state_bytes < h->state_bytes || work_bytes < h->work_bytes)
        return fail(h, LBM_ESIZE, "buffer smaller than reported by lbm_set_grid");
    cudaGetDevice(&h->device);
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaDeviceGetAttribute");
    int64_t blocks = (h->N + lbm::kRedThreads - 1) / lbm::kRedThreads;
    int64_t cap = std::min<int64_t>(lbm::kMaxRedBlocks, 4LL * sms);
    h->red_blocks = (int)std::max<int64_t>(1, std::min(blocks, cap));
    h->buf[0] = buf_a;
    h->buf[1] = buf_b;
    h->work = static_cast<char *>(work);
    h->stream = static_cast<cudaStream_t>(stream);
    h->cur = 0;
    h->has_state = false;
    e = cudaMemsetAsync(h->work + lbm::kWorkStatus, 0, sizeof(int), h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemsetAsync(status)");
    h->bound = true;
    return LBM_OK;
}

int lbm_set_macro(lbm_handle h, const float *rho, const float *u, const float *T)
{
    if (!h) return LBM_EINVAL;
    if (!h->bound) return fail(h, LBM_ESTATE, "lbm_bind must precede lbm_set_macro");
    if (!rho || !u || !T) return fail(h, LBM_EINVAL, "null field pointer");
    DeviceGuard g(h->device);
    Args a = make_args(h);
    a.dst = static_cast<float *>(h->buf[0]);
    a.in0 = rho;
    a.in1 = u;
    a.in2 = T;
    cudaError_t e = launch(h, Op::Init, a);
    if (e != cudaSuccess) return cuda_fail(h, e, "init kernel");
    h->cur = 0;
    h->steps = 0;
    h->has_state = true;
    return LBM_OK;
}

int lbm_step(lbm_handle h, int64_t k)
{
    if (!h) return LBM_EINVAL;
    if (k < 0) return fail(h, LBM_EINVAL, "k must be >= 0");
    if (!h->has_state) return fail(h, LBM_ESTATE, "no state: call lbm_set_macro or lbm_set_state");
    DeviceGuard g(h->device);
    Args a = make_args(h);
    for (int64_t s = 0; s < k; ++s) {
        a.src = static_cast<const float *>(h->buf[h->cur]);
        a.dst = static_cast<float *>(h->buf[h->cur ^ 1]);
        cudaError_t e = launch(h, Op::Step, a);
        if (e != cudaSuccess) return cuda_fail(h, e, "step kernel");
        h->cur ^= 1;
        ++h->steps;
    }
    return LBM_OK;
}

int lbm_get_moments(lbm_handle h, float *rho, float *u, float *T)
{
    if (!h) return LBM_EINVAL;
    if (!h->has_state) return fail(h, LBM_ESTATE, "no state");
    if (!rho || !u || !T) return fail(h, LBM_EINVAL, "null field pointer");
    DeviceGuard g(h->device);
    Args a = make_args(h);
    a.src = static_cast<const float *>(h->buf[h->cur]);
    a.out0 = rho;
    a.out1 = u;
    a.out2 = T;
    cudaError_t e = launch(h, Op::Moments, a);
    if (e != cudaSuccess) return cuda_fail(h, e, "moments kernel");
    return LBM_OK;
}

int lbm_conservation(lbm_handle h, double *out)
{
    if (!h) return LBM_EINVAL;
    if (!h->has_state) return fail(h, LBM_ESTATE, "no state");
    if (!out) return fail(h, LBM_EINVAL, "null output");
    DeviceGuard g(h->device);
    Args a = make_args(h);
    a.src = static_cast<const float *>(h->buf[h->cur]);
    cudaError_t e = launch(h, Op::Conserve, a);
    if (e != cudaSuccess) return cuda_fail(h, e, "conservation kernel");
    double *result = reinterpret_cast<double *>(h->work + lbm::kWorkResult);
    ++h->launches;
    k_finalize<<<1, lbm::kRedThreads, 0, h->stream>>>(a.partials, h->red_blocks, result);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "finalize kernel");
    double res[lbm::kRedSlots];
    int status = 0;
    e = cudaMemcpyAsync(res, result, sizeof(res), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&status, h->work + lbm::kWorkStatus, sizeof(int), cudaMemcpyDeviceToHost,
                            h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "conservation readback");
    out[0] = res[0];
    for (int d = 0; d < h->D; ++d) out[1 + d] = res[1 + d];
    out[1 + h->D] = res[4];
    out[2 + h->D] = res[5];
    if (status & 2) return fail(h, LBM_ETIMEOUT, "a staged step gave up waiting for its copies");
    if (status) return fail(h, LBM_ENONFINITE, "a step produced a non-finite or non-positive rho or T");
    return LBM_OK;
}

int lbm_get_state(lbm_handle h, float *ft, float *fr)
{
    if (!h) return LBM_EINVAL;
    if (!h->has_state) return fail(h, LBM_ESTATE, "no state");
    if (!ft || (h->Qr && !fr)) return fail(h, LBM_EINVAL, "null output");
    DeviceGuard g(h->device);
    Args a = make_args(h);
    a.src = static_cast<const float *>(h->buf[h->cur]);
    a.out0 = ft;
    a.out1 = fr;
    cudaError_t e = launch(h, Op::GetState, a);
    if (e != cudaSuccess) return cuda_fail(h, e, "get_state kernel");
    return LBM_OK;
}

int lbm_sample_state(lbm_handle h, const int64_t *nodes, int count, float *out)
{
    if (!h) return LBM_EINVAL;
    if (!h->has_state) return fail(h, LBM_ESTATE, "no state");
    if (!nodes || !out || count < 1 || count > (1 << 20)) return fail(h, LBM_EINVAL, "bad sample");
    DeviceGuard g(h->device);
    Args a = make_args(h);
    a.src = static_cast<const float *>(h->buf[h->cur]);
    a.nodes = nodes;
    a.count = count;
    a.out0 = out;
    cudaError_t e = launch(h, Op::Sample, a);
    if (e != cudaSuccess) return cuda_fail(h, e, "sample kernel");
    return LBM_OK;
}

int lbm_set_state(lbm_handle h, const float *ft, const float *fr)
{
    if (!h) return LBM_EINVAL;
    if (!h->bound) return fail(h, LBM_ESTATE, "lbm_bind must precede lbm_set_state");
    if (!ft || (h->Qr && !fr)) return fail(h, LBM_EINVAL, "null input");
    DeviceGuard g(h->device);
    Args a = make_args(h);
    a.dst = static_cast<float *>(h->buf[0]);
    a.in0 = ft;
    a.in1 = fr;
    cudaError_t e = launch(h, Op::SetState, a);
    if (e != cudaSuccess) return cuda_fail(h, e, "set_state kernel");
    h->cur = 0;
    h->steps = 0;
    h->has_state = true;
    return LBM_OK;
}

int lbm_status(lbm_handle h)
{
    if (!h) return LBM_EINVAL;
    if (!h->bound) return LBM_OK;
    DeviceGuard g(h->device);
    int status = 0;
    cudaError_t e = cudaMemcpyAsync(&status, h->work + lbm::kWorkStatus, sizeof(int),
                                    cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "status readback");
    if (status & 2) return LBM_ETIMEOUT;
    return status ? LBM_ENONFINITE : LBM_OK;
}

int64_t lbm_steps(lbm_handle h) { return h ? h->steps : -1; }

int64_t lbm_launch_count(lbm_handle h) { return h ? h->launches : -1; }

const char *lbm_last_error(lbm_handle h) { return h ? h->err.c_str() : "null handle"; }

void lbm_destroy(lbm_handle h) { delete h; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Conservation sums without any caller-provided scratch.
//
// lbm_conservation needs the work buffer bound with lbm_bind for its
// per-block partial sums.  Some callers cannot provide one: a host
// application that hands this library a state buffer but owns all device
// memory itself (its allocator has reserved the GPU, or its memory budget is
// fixed before the run), or a checker that inspects a saved state outside
// any bound solver.  lbm_conservation_noalloc serves them: its scratch is the
// file-scope array below, which every GPU that loads this library holds until
// the process exits, and it never calls cudaMalloc, cudaFree or any other
// allocating routine.

namespace {

constexpr int kNoAllocMaxBlocks = 1024;  // reduction blocks the array can hold
constexpr int kNoAllocMaxDevices = 64;

// kNoAllocMaxBlocks partial records, then one record for the final sums
// (kRedSlots doubles each): 65,600 bytes.  In host code this name is only a
// stand-in for the device array; its device address comes from
// cudaGetSymbolAddress.
static __device__ __align__(256) double g_noalloc_scratch[(kNoAllocMaxBlocks + 1) * lbm::kRedSlots];

std::mutex g_noalloc_mu;
double *g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device, looked up once
// per device (with that device current) and cached for the life of the
// process.  A cudaDeviceReset destroys the context the address belongs to,
// so the cache is not valid across one (the header says so).
cudaError_t noalloc_scratch(int dev, double **out)
{
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int lbm_conservation_noalloc(lbm_handle h, const void *state, void *stream, double *out)
{
    if (!h) return LBM_EINVAL;
    if (!h->grid_set) return fail(h, LBM_ESTATE, "lbm_set_grid must precede lbm_conservation_noalloc");
    if (!state || !out) return fail(h, LBM_EINVAL, "null state or output");
    if (!aligned256(state)) return fail(h, LBM_EINVAL, "state must be 256-byte aligned");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGetDevice");
    if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(h, LBM_EINVAL, "device ordinal too large");
    // The state must be device (or managed) memory of the current device: a
    // host pointer or another GPU's buffer would make the reduction kernel
    // fault.  This query reads only the driver's host-side records.
    cudaPointerAttributes attr{};
    e = cudaPointerGetAttributes(&attr, state);
    if (e != cudaSuccess) {
        cudaGetLastError();  // clear the (non-sticky) error this query left behind
        return fail(h, LBM_EINVAL, "state is not a CUDA device pointer");
    }
    if ((attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged) ||
        attr.device != dev)
        return fail(h, LBM_EINVAL, "state must be device memory of the current device");
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaDeviceGetAttribute");
    const int64_t want = std::min<int64_t>((h->N + lbm::kRedThreads - 1) / lbm::kRedThreads, 4LL * sms);
    const int blocks = (int)std::max<int64_t>(1, want);
    if (blocks > kNoAllocMaxBlocks)
        return fail(h, LBM_ESIZE, "the reduction needs " + std::to_string(blocks) +
                                      " blocks of scratch; the static array holds " +
                                      std::to_string(kNoAllocMaxBlocks));
    double *scratch = nullptr;
    e = noalloc_scratch(dev, &scratch);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGetSymbolAddress(g_noalloc_scratch)");

    // Each block overwrites all of its partial record and the final kernel
    // overwrites the result record, so nothing left by an earlier call is
    // read and nothing needs clearing first.
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Args a = make_args(h);
    a.src = static_cast<const float *>(state);
    a.partials = scratch;
    a.red_blocks = blocks;
    a.status = nullptr;
    switch (h->lattice) {
    case LBM_D1Q7: e = lbm::launch_d1q7(Op::Conserve, a, s); break;
    case LBM_D2Q37: e = lbm::launch_d2q37(Op::Conserve, a, s); break;
    case LBM_D2Q49: e = lbm::launch_d2q49(Op::Conserve, a, s); break;
    case LBM_D3Q343: e = lbm::launch_d3q343(Op::Conserve, a, s); break;
    default: e = cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "conservation kernel");
    double *result = scratch + (size_t)kNoAllocMaxBlocks * lbm::kRedSlots;
    k_finalize<<<1, lbm::kRedThreads, 0, s>>>(scratch, blocks, result);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "finalize kernel");
    h->launches += 2;
    double res[lbm::kRedSlots];
    e = cudaMemcpyAsync(res, result, sizeof(res), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(h, e, "conservation readback");
    out[0] = res[0];
    for (int d = 0; d < h->D; ++d) out[1 + d] = res[1 + d];
    out[1 + h->D] = res[4];
    out[2 + h->D] = res[5];
    return LBM_OK;
}
