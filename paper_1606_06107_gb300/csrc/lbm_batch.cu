// Ensembles of independent 1-D problems (D1Q7 + D1Q7, copy ends) advanced
// by one persistent launch: the lbm_batch_* part of the C ABI (include/lbm.h).
//
// Each resident block claims whole problems, longest first, from an atomic
// counter and runs all k steps of its problem with a block barrier between
// steps; the node update is the same device code as lbm_step's (k_step), so
// results are bit-identical to running each problem alone.  Loads use the
// L2-coherent path because the launch reads back what it wrote one step
// earlier.  A problem of L nodes keeps 2 x 14 x L floats live, so the
// resident problems (a few hundred) stay in the 126 MB L2 for their whole run.
// When the longest problem has at most 864 nodes, a second form keeps each
// problem's two buffers in shared memory for the whole run (k_batch_run_sm).
// A per-problem watch range limits which nodes may set its status word.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/lbm.h"
#include "lbm_step.cuh"

namespace lbm {
namespace {

constexpr int kD1 = 1;  // Lattice<1> = D1Q7

struct TubeDesc {    // one problem, indexed by its original position
    uint32_t base;   // first float of the problem in a state buffer
    int len;         // nodes
    int pitch;       // floats per population array (len rounded up to 32)
    int node_off;    // first node in the macro arrays
    float omega;     // BGK rate, with 1 - omega exact in float
    float cT;        // (D + n)/2
    float half_n;    // n/2
    float half_n_r2; // n r^2 / 2
    int watch_lo;    // nodes [watch_lo, watch_hi) set the status word
    int watch_hi;
};

struct BatchParams {
    const TubeDesc *tubes;
    const int *order;  // processing order (longest first)
    int count;
    float *buf[2];
    int cur;           // buffer holding the state at step 0
    long long steps;
    int *status;       // per problem
    int *counter;
    float r, r2, inv_r2, nu_scale, inv_m;
    float w[7], wr[7];
};

__device__ __forceinline__ Params<7> tube_params(const BatchParams &bp, const TubeDesc &d,
                                                 const float *src, float *dst)
{
    Params<7> p;
    p.src = src ? src + d.base : nullptr;
    p.dst = dst ? dst + d.base : nullptr;
    p.in0 = p.in1 = p.in2 = nullptr;
    p.out0 = p.out1 = p.out2 = nullptr;
    p.status = nullptr;
    p.partials = nullptr;
    p.S = d.pitch;
    p.N = d.len;
    p.X = d.len;
    p.Y = 1;
    p.Z = 1;
    p.pitch = d.pitch;
    p.bc0 = LBM_BC_COPY;
    p.bc1 = p.bc2 = LBM_BC_PERIODIC;
    p.r = bp.r;
    p.r2 = bp.r2;
    p.inv_r2 = bp.inv_r2;
    p.omega = d.omega;
    p.nu_scale = bp.nu_scale;
    p.cT = d.cT;
    p.half_n = d.half_n;
    p.half_n_r2 = d.half_n_r2;
    p.inv_m = bp.inv_m;
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        p.w[i] = bp.w[i];
        p.wr[i] = bp.wr[i];
    }
    return p;
}

// One node of one problem: the body of k_step<D1Q7, rot, MODE> with
// L2-coherent loads (CG = 1) or plain loads from shared memory (CG = 2).
template <int MODE, int CG = 1>
__device__ __forceinline__ void batch_node(const Params<7> &p, const TubeDesc &d, int x)
{
    const Offsets o = node_offsets<1>(p, x, 0, 0);
    float g[7], h[7];
    load_node<kD1, true, MODE, CG>(p, o, g, h);
    const Moments m = node_moments<kD1, true>(p, g, h);
    if ((!(m.rho > 0.f) || !(m.T > 0.f) || !(fabsf(m.T) < 3.0e38f)) && x >= d.watch_lo &&
        x < d.watch_hi)
        atomicOr(p.status, 1);
    collide_store<kD1>(p, o.self(), g, m, [&](auto ic, float gi) {
        return transport<kD1, MODE, decltype(ic)::value, CG>(p, o, gi);
    });
    float adv[7];
    rot_advect<1, CG>(p, o, h, m, adv);
    rot_store(p, o.self(), h, m, adv);
}

template <int MODE>
__global__ void __launch_bounds__(1024) k_batch_run(const BatchParams bp)
{
    __shared__ int claim;
    for (;;) {
        if (threadIdx.x == 0) claim = atomicAdd(bp.counter, 1);
        __syncthreads();
        const int slot = claim;
        __syncthreads();  // every thread has read `claim` before it is reused
        if (slot >= bp.count) return;
        const int k = bp.order[slot];
        const TubeDesc d = bp.tubes[k];
        int cur = bp.cur;
        for (long long s = 0; s < bp.steps; ++s) {
            Params<7> p = tube_params(bp, d, bp.buf[cur], bp.buf[cur ^ 1]);
            p.status = bp.status + k;
            for (int x = threadIdx.x; x < d.len; x += blockDim.x) batch_node<MODE>(p, d, x);
            cur ^= 1;
            __syncthreads();  // step s+1 reads neighbours written in step s
        }
    }
}

// The same schedule for problems whose two state buffers fit in shared
// memory (14 x pitch floats each): the block copies its problem in, steps
// it between two shared-memory buffers (a step is then bound by shared-
// memory latency instead of the L2 round trip of each neighbour load), and
// copies the result to the global buffer the other form would end in.  The
// node update is the same code, so the results are the same bits.
template <int MODE>
__global__ void __launch_bounds__(1024) k_batch_run_sm(const BatchParams bp)
{
    extern __shared__ float sm[];
    __shared__ int claim;
    for (;;) {
        if (threadIdx.x == 0) claim = atomicAdd(bp.counter, 1);
        __syncthreads();
        const int slot = claim;
        __syncthreads();  // every thread has read `claim` before it is reused
        if (slot >= bp.count) return;
        const int k = bp.order[slot];
        const TubeDesc d = bp.tubes[k];
        const int n = 14 * d.pitch;
        float *a = sm, *c = sm + n;  // a holds the current state
        const float *in = bp.buf[bp.cur] + d.base;
        for (int e = threadIdx.x; e < n; e += blockDim.x) a[e] = __ldcg(in + e);
        __syncthreads();
        for (long long s = 0; s < bp.steps; ++s) {
            Params<7> p = tube_params(bp, d, nullptr, nullptr);
            p.src = a;
            p.dst = c;
            p.status = bp.status + k;
            for (int x = threadIdx.x; x < d.len; x += blockDim.x) batch_node<MODE, 2>(p, d, x);
            float *t = a;
            a = c;
            c = t;
            __syncthreads();  // step s+1 reads neighbours written in step s
        }
        float *out = bp.buf[bp.cur ^ (int)(bp.steps & 1)] + d.base;
        for (int e = threadIdx.x; e < n; e += blockDim.x) out[e] = a[e];
        // the claim's barriers order these reads before the next copy-in
    }
}

template <int MODE>
__global__ void __launch_bounds__(kBlockX) k_batch_init(const BatchParams bp, const float *rho,
                                                        const float *u, const float *T)
{
    const TubeDesc d = bp.tubes[blockIdx.y];
    const int x = blockIdx.x * kBlockX + threadIdx.x;
    if (x >= d.len) return;
    Params<7> p = tube_params(bp, d, nullptr, bp.buf[bp.cur]);
    p.in0 = rho + d.node_off;
    p.in1 = u + d.node_off;
    p.in2 = T + d.node_off;
    init_node<kD1, true, MODE>(p, x, 0, 0);
}

template <int MODE>
__global__ void __launch_bounds__(kBlockX) k_batch_moments(const BatchParams bp, float *rho,
                                                           float *u, float *T)
{
    const TubeDesc d = bp.tubes[blockIdx.y];
    const int x = blockIdx.x * kBlockX + threadIdx.x;
    if (x >= d.len) return;
    Params<7> p = tube_params(bp, d, bp.buf[bp.cur], nullptr);
    p.out0 = rho + d.node_off;
    p.out1 = u + d.node_off;
    p.out2 = T + d.node_off;
    moments_node<kD1, true, MODE>(p, x, 0, 0);
}

// D1Q7 constants solved in double precision (lbm_lattice_info).
void d1q7(double *r, double w[7])
{
    int e[343 * 3];
    lbm_lattice_info(LBM_D1Q7, r, e, w);
}

size_t align256(size_t n) { return (n + 255) / 256 * 256; }

// Largest shared-memory state (two buffers of the longest problem) for
// which a run takes the shared-memory form: 96 KB keeps at least two blocks
// per SM (problems of up to 864 nodes).
#ifndef LBM_BATCH_SMEM_MAX
#define LBM_BATCH_SMEM_MAX (96 * 1024)
#endif

}  // namespace
}  // namespace lbm

using lbm::BatchParams;
using lbm::TubeDesc;

struct lbm_batch_ctx {
    int count = 0, mode = LBM_MODE_STREAM, m_fd = 1;
    double r = 0.0, w[7] = {};
    std::vector<TubeDesc> tubes;
    std::vector<int> order;
    int max_len = 0;
    int sm_bytes = 0;  // > 0: runs take the shared-memory form with this much per block
    int64_t total_nodes = 0;
    size_t state_floats = 0;
    size_t off_tubes = 0, off_order = 0, off_status = 0, off_counter = 0, work_bytes = 0;
    bool bound = false, has_state = false;
    float *buf[2] = {nullptr, nullptr};
    char *work = nullptr;
    cudaStream_t stream = nullptr;
    int cur = 0;
    int threads = 256;
    int blocks_per_sm = 0;  // resident blocks per SM of the persistent grid (0 = max)
    int64_t launches = 0;
    std::string err;
    struct Cached {
        cudaGraphExec_t exec = nullptr;
        long long steps = -1;
        int cur = -1, threads = -1, bps = -1;
    } graphs[2];
    int next_graph = 0;
};

namespace {

int bfail(lbm_batch b, int code, const std::string &msg)
{
    if (b) b->err = msg;
    return code;
}

int bcuda(lbm_batch b, cudaError_t e, const char *where)
{
    return bfail(b, LBM_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

BatchParams batch_params(const lbm_batch_ctx *b, long long steps)
{
    BatchParams bp{};
    bp.tubes = reinterpret_cast<const TubeDesc *>(b->work + b->off_tubes);
    bp.order = reinterpret_cast<const int *>(b->work + b->off_order);
    bp.count = b->count;
    bp.buf[0] = b->buf[0];
    bp.buf[1] = b->buf[1];
    bp.cur = b->cur;
    bp.steps = steps;
    bp.status = reinterpret_cast<int *>(b->work + b->off_status);
    bp.counter = reinterpret_cast<int *>(b->work + b->off_counter);
    const double m = (b->mode == LBM_MODE_FD) ? b->m_fd : 1.0;
    bp.r = (float)b->r;
    bp.r2 = bp.r * bp.r;
    bp.inv_r2 = 1.0f / (bp.r * bp.r);
    bp.nu_scale = (float)(1.0 / (m * b->r));
    bp.inv_m = (float)(1.0 / m);
    for (int j = 0; j < 7; ++j) {
        bp.w[j] = (float)b->w[j];
        bp.wr[j] = (float)b->w[j];
    }
    return bp;
}

bool aligned(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 255u) == 0; }

// The persistent kernel of a run: the shared-memory form when the longest
// problem fits (sm_bytes > 0), else the global-memory form.
const void *run_kernel(const lbm_batch_ctx *b)
{
    if (b->sm_bytes > 0)
        return (b->mode == LBM_MODE_FD) ? (const void *)lbm::k_batch_run_sm<1>
                                        : (const void *)lbm::k_batch_run_sm<0>;
    return (b->mode == LBM_MODE_FD) ? (const void *)lbm::k_batch_run<1>
                                    : (const void *)lbm::k_batch_run<0>;
}

// Resident-block grid of the persistent kernel for `threads` per block.
cudaError_t persistent_grid(const lbm_batch_ctx *b, int threads, int bps, int *grid)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const void *fn = run_kernel(b);
    if (b->sm_bytes > 0)
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, b->sm_bytes);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, b->sm_bytes);
    if (e != cudaSuccess) return e;
    per_sm = std::max(1, per_sm);
    if (bps > 0) per_sm = std::min(per_sm, bps);
    *grid = per_sm * sms;
    return cudaSuccess;
}

// The graph of one run: reset the claim counter, then the persistent kernel.
int build_graph(lbm_batch b, long long steps, cudaGraphExec_t *exec)
{
    int grid = 0;
    cudaError_t e = persistent_grid(b, b->threads, b->blocks_per_sm, &grid);
    if (e != cudaSuccess) return bcuda(b, e, "occupancy query");
    cudaGraph_t g = nullptr;
    e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return bcuda(b, e, "cudaGraphCreate");
    cudaMemsetParams ms{};
    ms.dst = b->work + b->off_counter;
    ms.value = 0;
    ms.elementSize = 4;
    ms.width = 1;
    ms.height = 1;
    ms.pitch = 4;
    cudaGraphNode_t n_reset = nullptr, n_run = nullptr;
    e = cudaGraphAddMemsetNode(&n_reset, g, nullptr, 0, &ms);
    BatchParams bp = batch_params(b, steps);
    void *args[] = {&bp};
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void *>(run_kernel(b));
    kp.gridDim = dim3(grid);
    kp.blockDim = dim3(b->threads);
    kp.sharedMemBytes = (unsigned)b->sm_bytes;
    kp.kernelParams = args;
    if (e == cudaSuccess) e = cudaGraphAddKernelNode(&n_run, g, &n_reset, 1, &kp);
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bcuda(b, e, "graph build");
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_batch_create(int count, const int64_t *lengths, const int *n, const double *tau, int mode,
                     int m_fd, lbm_batch *out)
{
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    if (count < 1 || count > 65535 || !lengths || !n || !tau) return LBM_EINVAL;
    if (mode != LBM_MODE_STREAM && mode != LBM_MODE_FD) return LBM_EINVAL;
    if (mode == LBM_MODE_FD && m_fd < 1) return LBM_EINVAL;
    lbm_batch b = new lbm_batch_ctx();
    b->count = count;
    b->mode = mode;
    b->m_fd = (mode == LBM_MODE_FD) ? m_fd : 1;
    lbm::d1q7(&b->r, b->w);
    const double m = b->m_fd;
    b->tubes.resize(count);
    size_t base = 0;
    int64_t node = 0;
    for (int k = 0; k < count; ++k) {
        if (lengths[k] < 1 || lengths[k] > (1 << 30) || n[k] < 0 || !(tau[k] > 0.0) ||
            !std::isfinite(tau[k])) {
            delete b;
            return LBM_EINVAL;
        }
        TubeDesc &d = b->tubes[k];
        d.len = (int)lengths[k];
        d.pitch = (d.len + 31) / 32 * 32;
        d.base = (uint32_t)base;
        d.node_off = (int)node;
        // omega with an exact 1 - omega, as for lbm_handle
        const float om = (float)(1.0 / (m * tau[k]));
        const float keep = (float)(1.0 - (double)om);
        d.omega = (float)(1.0 - (double)keep);
        d.cT = (float)(0.5 * (1 + n[k]));
        d.half_n = (float)(0.5 * n[k]);
        d.half_n_r2 = (float)(0.5 * n[k] * b->r * b->r);
        d.watch_lo = 0;
        d.watch_hi = d.len;
        base += (size_t)14 * d.pitch;
        node += d.len;
        b->max_len = std::max(b->max_len, d.len);
        if (base > 0x7fffffffULL || node > 0x7fffffffLL) {
            delete b;
            return LBM_ESIZE;
        }
    }
    b->state_floats = base;
    b->total_nodes = node;
    const size_t sm = (size_t)2 * 14 * ((b->max_len + 31) / 32 * 32) * sizeof(float);
    b->sm_bytes = (sm <= (size_t)LBM_BATCH_SMEM_MAX) ? (int)sm : 0;
    b->order.resize(count);
    std::iota(b->order.begin(), b->order.end(), 0);
    std::stable_sort(b->order.begin(), b->order.end(),
                     [&](int a, int c) { return b->tubes[a].len > b->tubes[c].len; });
    b->off_tubes = 0;
    b->off_order = lbm::align256(sizeof(TubeDesc) * count);
    b->off_status = b->off_order + lbm::align256(sizeof(int) * count);
    b->off_counter = b->off_status + lbm::align256(sizeof(int) * count);
    b->work_bytes = b->off_counter + 256;
    *out = b;
    return LBM_OK;
}

int lbm_batch_set_problems(lbm_batch b, const int *n, const double *tau)
{
    if (!b) return LBM_EINVAL;
    if (!n || !tau) return bfail(b, LBM_EINVAL, "null n or tau");
    for (int k = 0; k < b->count; ++k)
        if (n[k] < 0 || !(tau[k] > 0.0) || !std::isfinite(tau[k]))
            return bfail(b, LBM_EINVAL, "bad n or tau");
    const double m = b->m_fd;
    for (int k = 0; k < b->count; ++k) {
        TubeDesc &d = b->tubes[k];
        const float om = (float)(1.0 / (m * tau[k]));
        const float keep = (float)(1.0 - (double)om);
        d.omega = (float)(1.0 - (double)keep);
        d.cT = (float)(0.5 * (1 + n[k]));
        d.half_n = (float)(0.5 * n[k]);
        d.half_n_r2 = (float)(0.5 * n[k] * b->r * b->r);
    }
    if (b->bound) {
        cudaError_t e = cudaMemcpyAsync(b->work + b->off_tubes, b->tubes.data(),
                                        sizeof(TubeDesc) * b->count, cudaMemcpyHostToDevice,
                                        b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "table upload");
        b->has_state = false;
    }
    return LBM_OK;
}

int lbm_batch_set_watch(lbm_batch b, const int *lo, const int *hi)
{
    if (!b) return LBM_EINVAL;
    if ((lo == nullptr) != (hi == nullptr)) return bfail(b, LBM_EINVAL, "lo and hi go together");
    for (int k = 0; lo && k < b->count; ++k)
        if (lo[k] < 0 || lo[k] > hi[k] || hi[k] > b->tubes[k].len)
            return bfail(b, LBM_EINVAL, "watch range outside the problem");
    for (int k = 0; k < b->count; ++k) {
        b->tubes[k].watch_lo = lo ? lo[k] : 0;
        b->tubes[k].watch_hi = lo ? hi[k] : b->tubes[k].len;
    }
    if (b->bound) {
        cudaError_t e = cudaMemcpyAsync(b->work + b->off_tubes, b->tubes.data(),
                                        sizeof(TubeDesc) * b->count, cudaMemcpyHostToDevice,
                                        b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "table upload");
    }
    return LBM_OK;
}

int lbm_batch_sizes(lbm_batch b, size_t *state_bytes, size_t *work_bytes, int64_t *total_nodes)
{
    if (!b) return LBM_EINVAL;
    if (state_bytes) *state_bytes = sizeof(float) * b->state_floats;
    if (work_bytes) *work_bytes = b->work_bytes;
    if (total_nodes) *total_nodes = b->total_nodes;
    return LBM_OK;
}

int lbm_batch_bind(lbm_batch b, void *buf_a, void *buf_b, size_t state_bytes, void *work,
                   size_t work_bytes, void *stream)
{
    if (!b) return LBM_EINVAL;
    if (!buf_a || !buf_b || !work || buf_a == buf_b) return bfail(b, LBM_EINVAL, "bad buffers");
    if (!aligned(buf_a) || !aligned(buf_b) || !aligned(work))
        return bfail(b, LBM_EINVAL, "buffers must be 256-byte aligned");
    if (state_bytes < sizeof(float) * b->state_floats || work_bytes < b->work_bytes)
        return bfail(b, LBM_ESIZE, "buffer smaller than reported by lbm_batch_sizes");
    b->buf[0] = static_cast<float *>(buf_a);
    b->buf[1] = static_cast<float *>(buf_b);
    b->work = static_cast<char *>(work);
    b->stream = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(b->work + b->off_tubes, b->tubes.data(),
                                    sizeof(TubeDesc) * b->count, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->work + b->off_order, b->order.data(), sizeof(int) * b->count,
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(b->work + b->off_status, 0, sizeof(int) * b->count, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "table upload");
    for (auto &c : b->graphs) {
        if (c.exec) cudaGraphExecDestroy(c.exec);
        c = lbm_batch_ctx::Cached{};
    }
    b->bound = true;
    b->has_state = false;
    b->cur = 0;
    return LBM_OK;
}

int lbm_batch_set_macro(lbm_batch b, const float *rho, const float *u, const float *T)
{
    if (!b) return LBM_EINVAL;
    if (!b->bound) return bfail(b, LBM_ESTATE, "lbm_batch_bind must precede lbm_batch_set_macro");
    if (!rho || !u || !T) return bfail(b, LBM_EINVAL, "null field pointer");
    b->cur = 0;
    BatchParams bp = batch_params(b, 0);
    const dim3 grid((b->max_len + lbm::kBlockX - 1) / lbm::kBlockX, b->count);
    if (b->mode == LBM_MODE_FD)
        lbm::k_batch_init<1><<<grid, lbm::kBlockX, 0, b->stream>>>(bp, rho, u, T);
    else
        lbm::k_batch_init<0><<<grid, lbm::kBlockX, 0, b->stream>>>(bp, rho, u, T);
    ++b->launches;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemsetAsync(b->work + b->off_status, 0, sizeof(int) * b->count, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "batch init");
    b->has_state = true;
    return LBM_OK;
}

int lbm_batch_run(lbm_batch b, int64_t k)
{
    if (!b) return LBM_EINVAL;
    if (k < 0) return bfail(b, LBM_EINVAL, "k must be >= 0");
    if (!b->has_state) return bfail(b, LBM_ESTATE, "no state: call lbm_batch_set_macro");
    if (k == 0) return LBM_OK;
    lbm_batch_ctx::Cached *hit = nullptr;
    for (auto &c : b->graphs)
        if (c.exec && c.steps == k && c.cur == b->cur && c.threads == b->threads &&
            c.bps == b->blocks_per_sm)
            hit = &c;
    if (!hit) {
        hit = &b->graphs[b->next_graph];
        b->next_graph ^= 1;
        if (hit->exec) cudaGraphExecDestroy(hit->exec);
        *hit = lbm_batch_ctx::Cached{};
        const int rc = build_graph(b, k, &hit->exec);
        if (rc != LBM_OK) return rc;
        hit->steps = k;
        hit->cur = b->cur;
        hit->threads = b->threads;
        hit->bps = b->blocks_per_sm;
    }
    cudaError_t e = cudaGraphLaunch(hit->exec, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "cudaGraphLaunch");
    ++b->launches;
    b->cur ^= (int)(k & 1);
    return LBM_OK;
}

int lbm_batch_get_moments(lbm_batch b, float *rho, float *u, float *T)
{
    if (!b) return LBM_EINVAL;
    if (!b->has_state) return bfail(b, LBM_ESTATE, "no state");
    if (!rho || !u || !T) return bfail(b, LBM_EINVAL, "null field pointer");
    BatchParams bp = batch_params(b, 0);
    const dim3 grid((b->max_len + lbm::kBlockX - 1) / lbm::kBlockX, b->count);
    if (b->mode == LBM_MODE_FD)
        lbm::k_batch_moments<1><<<grid, lbm::kBlockX, 0, b->stream>>>(bp, rho, u, T);
    else
        lbm::k_batch_moments<0><<<grid, lbm::kBlockX, 0, b->stream>>>(bp, rho, u, T);
    ++b->launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bcuda(b, e, "batch moments");
    return LBM_OK;
}

int lbm_batch_status(lbm_batch b, int *status, int *n_bad)
{
    if (!b) return LBM_EINVAL;
    if (!b->bound) return bfail(b, LBM_ESTATE, "not bound");
    std::vector<int> host(b->count);
    cudaError_t e = cudaMemcpyAsync(host.data(), b->work + b->off_status, sizeof(int) * b->count,
                                    cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "status readback");
    int bad = 0;
    for (int k = 0; k < b->count; ++k) bad += host[k] != 0;
    if (status) std::copy(host.begin(), host.end(), status);
    if (n_bad) *n_bad = bad;
    return LBM_OK;
}

int lbm_batch_set_block(lbm_batch b, int threads, int blocks_per_sm)
{
    if (!b) return LBM_EINVAL;
    if (threads < 32 || threads > 1024 || threads % 32)
        return bfail(b, LBM_EINVAL, "threads must be a multiple of 32 in 32..1024");
    if (blocks_per_sm < 0) return bfail(b, LBM_EINVAL, "blocks_per_sm must be >= 0");
    b->threads = threads;
    b->blocks_per_sm = blocks_per_sm;
    return LBM_OK;
}

int lbm_batch_autotune(lbm_batch b, int64_t sample_steps, int *threads, int *blocks_per_sm)
{
    if (!b) return LBM_EINVAL;
    if (sample_steps < 1) return bfail(b, LBM_EINVAL, "sample_steps must be >= 1");
    if (!b->has_state) return bfail(b, LBM_ESTATE, "no state: call lbm_batch_set_macro");
    // Block size x resident blocks per SM: fewer resident problems keep more
    // of each one's state in L2, more blocks hide more latency.
    static const int cand_threads[] = {128, 256, 512, 1024};
    static const int cand_bps[] = {1, 2, 4, 0};
    cudaEvent_t t0, t1;
    cudaError_t e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    if (e != cudaSuccess) return bcuda(b, e, "cudaEventCreate");
    float best_ms = 0.f;
    int best_t = b->threads, best_b = b->blocks_per_sm;
    for (int c : cand_threads) {
        for (int bps : cand_bps) {
            b->threads = c;
            b->blocks_per_sm = bps;
            int rc = lbm_batch_run(b, sample_steps);  // builds the graph, warms up
            if (rc != LBM_OK) break;
            e = cudaEventRecord(t0, b->stream);
            rc = lbm_batch_run(b, sample_steps);
            if (rc != LBM_OK) break;
            if (e == cudaSuccess) e = cudaEventRecord(t1, b->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(t1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
            if (e != cudaSuccess) break;
            if (best_ms == 0.f || ms < best_ms) {
                best_ms = ms;
                best_t = c;
                best_b = bps;
            }
        }
        if (e != cudaSuccess) break;
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    b->threads = best_t;
    b->blocks_per_sm = best_b;
    if (threads) *threads = best_t;
    if (blocks_per_sm) *blocks_per_sm = best_b;
    if (e != cudaSuccess) return bcuda(b, e, "autotune timing");
    return LBM_OK;
}

int64_t lbm_batch_launch_count(lbm_batch b) { return b ? b->launches : -1; }

const char *lbm_batch_last_error(lbm_batch b) { return b ? b->err.c_str() : "null handle"; }

void lbm_batch_destroy(lbm_batch b)
{
    if (!b) return;
    for (auto &c : b->graphs)
        if (c.exec) cudaGraphExecDestroy(c.exec);
    delete b;
}

}  // extern "C"
