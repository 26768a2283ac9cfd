/*
 * lbm.h -- C ABI of the GB300 (sm_103a) decoupled Hermite-expansion lattice
 * Boltzmann library (liblbm.so).
 *
 * The method is Hu, Zhang & Geng, "A decoupled scheme based on the Hermite
 * expansion to construct lattice Boltzmann models for the compressible
 * Navier-Stokes equations with arbitrary specific heat ratio" (arXiv
 * 1606.06107).  Each lattice node carries
 *   - Q_t translational populations g_i (the paper's g_i, Eq. DisEvolI) on a
 *     4th-order Hermite lattice: D1Q7 (Table II used as a 1-D translational
 *     set), D2Q37 (Table I) or the tensor product D2Q49 = D1Q7 x D1Q7, and
 *   - Q_r = 7 rotational populations h_j (Eq. EvoEtaJ) on D1Q7 (Table II)
 *     when the number of rotational degrees of freedom n > 0 (Q_r = 0 for
 *     n = 0).  The specific-heat ratio is gamma = (D+n+2)/(D+n) (Sec. III).
 *
 * One step advances both populations: moments rho, u, T of the time-t
 * populations (Sec. V steps 3-4, Eq. T), 4th-order Hermite equilibria
 * (Sec. IV), BGK relaxation, and transport.  Two transport modes exist:
 *   LBM_MODE_STREAM  g is pulled exactly on the lattice, g_i(x,t) =
 *                    ft_i(x - e_i) with xi_i = r e_i and dt = dx/r (the time
 *                    mapping t = step/(X r) of Sec. VI); the stored ft is the
 *                    post-collision value; omega = 1/tau (tau in steps).
 *   LBM_MODE_FD      the paper's forward-Euler + third-order upwind scheme
 *                    for g (Eq. DisEvolSpaTiI) with dt = dx/(m r);
 *                    omega = 1/(m tau).
 * In both modes h is advected by the fluid velocity with the third-order
 * upwind scheme of Eq. DisEvolSpaTiJ at Courant number u dt/dx and relaxed
 * toward h^eq(T).
 *
 * Units are the paper's dimensionless ones (Eq. DDF, theta0 = 1): P = rho T.
 *
 * Population order: velocities sorted by (ez, ey, ex) ascending; for D1Q7
 * index i has e = i - 3; for D2Q49 index i = (ey+3)*7 + (ex+3); for D2Q37
 * the D2Q49 order with the 12 velocities |e| in {(2,2),(2,3),(3,2)}
 * removed.  Rotational index j has eta_j = r (j - 3).
 *
 * Memory ownership: the library never allocates device memory.  The caller
 * allocates two state buffers and one work buffer of the sizes reported by
 * lbm_set_grid (any allocator; 256-byte alignment required) and binds them
 * with lbm_bind.  The handle owns host memory only.
 *
 * Field layout for lbm_set_macro / lbm_get_moments: float32 device arrays,
 * x fastest, unpadded, N = X*Y*Z entries; u is structure-of-arrays,
 * u[a*N + node] for axis a < D.
 *
 * Errors: every call returns an lbm_status; lbm_last_error gives a message.
 * Kernels never trap: a non-finite or non-positive rho or T found by a step
 * sets a sticky device flag that lbm_status and lbm_conservation report as
 * LBM_ENONFINITE.
 *
 * Threading: a handle is used by one host thread at a time.  Work is
 * enqueued on the stream given to lbm_bind; calls documented as
 * "synchronizing" wait for that stream.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx *lbm_handle;

enum lbm_lattice { LBM_D1Q7 = 1, LBM_D2Q37 = 2, LBM_D2Q49 = 3, LBM_D3Q343 = 4 };
enum lbm_bc { LBM_BC_PERIODIC = 0, LBM_BC_COPY = 1 };
enum lbm_mode { LBM_MODE_STREAM = 0, LBM_MODE_FD = 1 };
enum lbm_status {
    LBM_OK = 0,
    LBM_EINVAL = -1,     /* bad argument */
    LBM_ESIZE = -2,      /* grid or buffer size out of range */
    LBM_ECUDA = -3,      /* a CUDA runtime call failed */
    LBM_ENONFINITE = -4, /* a step produced non-finite or non-positive rho/T */
    LBM_ETIMEOUT = -5,   /* reserved: a bounded device wait gave up */
    LBM_ESTATE = -6      /* call out of order (e.g. step before bind) */
};

/* Create a solver.  D in {1,2,3}; lattice one of lbm_lattice with dimension
 * D; n >= 0 rotational degrees of freedom (gamma = (D+n+2)/(D+n), Sec. III);
 * tau > 0 relaxation time in lattice steps (Eq. DisEvolI/EvoEtaJ).  The
 * lattice scaling factor r and weights (Tables I, II) are solved on the host
 * in double precision from the Gauss-Hermite moment equations and rounded
 * once to float.  Mode defaults to LBM_MODE_STREAM.  LBM_D3Q343 (D = 3, the
 * tensor product D1Q7 x D1Q7 x D1Q7) runs in LBM_MODE_STREAM only. */
int lbm_create(int D, int lattice, int n, double tau, lbm_handle *out);

/* Select the transport mode (lbm_mode) and, for LBM_MODE_FD, the number m
 * >= 1 of forward-Euler sub-steps per lattice time dx/r (Eq. DisEvolSpaTiI).
 * Must be called before lbm_set_grid. */
int lbm_set_mode(lbm_handle h, int mode, int m_fd);

/* Storage of the populations in HBM (before lbm_set_grid).  LBM_STORE_F32
 * (default) keeps float32 values.  LBM_STORE_F16 / LBM_STORE_BF16 keep the
 * relative deviation from the rest equilibrium, d_i = f_i / w_i - 1, as IEEE
 * half / bfloat16, halving the bytes per step; all arithmetic stays float32
 * and the temperature is recovered from the total energy with its kinetic
 * part subtracted in double precision (Eq. T).  The reduced precision
 * changes results by the storage rounding (about 2^-11 resp. 2^-8 of d_i
 * per step).
 *
 * LBM_STORE_F16_NODE / LBM_STORE_BF16_NODE keep the deviation from a
 * per-node reference equilibrium instead, so the 16 bits resolve the
 * departure from the node's own local equilibrium rather than from rest.
 * Each node stores a reference record of four floats after the populations
 * (16 bytes per node, 14 % more bytes per step on D2Q49 + D1Q7):
 * (rho - 1, rho (T - 1) / 2, rho r u_x, rho r u_y) of the moments at which
 * the node last collided (set_macro: the initial fields; set_state: rest).  A
 * translational value is stored as s_i = f_i / w_i - R_i with the terms of
 * the Hermite equilibrium of Sec. IV of first order in u and of up to second
 * order in t = T - 1: R_i = rho (1 + xi_i.u + t (|xi_i|^2 - D) / 2)
 * + (rho t)^2 (|xi_i|^4 - 2 (D+2) |xi_i|^2 + D (D+2)) / 8, and a rotational value
 * as s_j = h_j / w_j - h_j^eq(T) / w_j (its full equilibrium, which depends
 * on T only); a pulled value is decoded with the record of the node it was
 * pulled from.  Writer and reader evaluate R from the same stored floats
 * with the same fused operations, so the reference cancels exactly.
 * LBM_MODE_STREAM and the 1-D and 2-D lattices only (lbm_set_grid returns
 * LBM_EINVAL otherwise). */
enum lbm_storage {
    LBM_STORE_F32 = 0,
    LBM_STORE_F16 = 1,
    LBM_STORE_BF16 = 2,
    LBM_STORE_F16_NODE = 3,
    LBM_STORE_BF16_NODE = 4
};
int lbm_set_storage(lbm_handle h, int storage);

/* Set the grid: shape[0..D-1] = X (fastest), Y, Z, each >= 1 (Y, Z <= 65535);
 * bc[0..D-1] per-axis boundary (periodic wrap, or copy = zero-gradient
 * clamp to the edge node, the paper's "open" boundary of Sec. VI).  Returns
 * the bytes needed for each of the two state buffers and for the work
 * buffer. */
int lbm_set_grid(lbm_handle h, const int64_t *shape, const int *bc,
                 size_t *state_bytes, size_t *work_bytes);

/* Bind caller-owned device memory: two state buffers (ping-pong) of
 * state_bytes each, a work buffer of work_bytes, and the CUDA stream
 * (cudaStream_t, NULL = legacy default) all later work is enqueued on.
 * Clears the sticky status flag (asynchronously, on that stream). */
int lbm_bind(lbm_handle h, void *buf_a, void *buf_b, size_t state_bytes, void *work,
             size_t work_bytes, void *stream);

/* Equilibrium initial state from the macroscopic fields (device pointers,
 * layout above): h_j = h_j^eq(T); in STREAM mode the stored ft is the pull
 * pre-image ft_i(x) = g_i^eq(m0(bc(x + e_i))), in FD mode ft_i = g_i^eq(m0(x)).
 * Asynchronous.  Resets the step counter. */
int lbm_set_macro(lbm_handle h, const float *rho, const float *u, const float *T);

/* Advance k >= 0 steps (Sec. V steps 1-5): one fused kernel launch per step.
 * Asynchronous. */
int lbm_step(lbm_handle h, int64_t k);

/* rho, u, T of the current state (Sec. V steps 3-4, Eq. T) into device
 * arrays (layout above).  Asynchronous. */
int lbm_get_moments(lbm_handle h, float *rho, float *u, float *T);

/* Global diagnostics of the current state, accumulated in double precision
 * with a fixed reduction order: out[0] = sum rho, out[1..D] = sum rho u_a,
 * out[D+1] = sum rho (E + u^2/2) (the total energy of Eq. Total),
 * out[D+2] = max over nodes of |sum_j h_j - 1| (Eq. FFeqRhoEta).  out is a
 * HOST pointer to D+3 doubles.  Synchronizing.  Returns LBM_ENONFINITE if the
 * sticky flag is set (out is still written). */
int lbm_conservation(lbm_handle h, double *out);

/* The sums of lbm_conservation for callers that cannot provide device
 * scratch memory (the paper has no counterpart; this is a library service).
 * A host application that owns all device memory itself -- its allocator has
 * reserved the GPU, or its memory budget is fixed before the run -- can pass
 * a state buffer here without binding a work buffer.  The per-block partial
 * sums live in a static device array inside the library (65,600 bytes, held
 * on every GPU that loads the library until the process exits); nothing is
 * allocated.
 *   state  device pointer to one state buffer in the layout lbm_set_grid
 *          describes (256-byte aligned), device or managed memory of the
 *          current device (checked on the host with
 *          cudaPointerGetAttributes; anything else is LBM_EINVAL).  For a bound
 *          handle, the current state is buf_a after an even number of steps
 *          since lbm_set_macro / lbm_set_state and buf_b after an odd number.
 *   stream cudaStream_t the work is enqueued on (NULL = legacy default).
 *   out    HOST pointer to D+3 doubles, filled as by lbm_conservation.
 * Needs lbm_set_grid, not lbm_bind; does not read the sticky status flag.
 * Synchronizing (waits for `stream`).  The first call on each device looks
 * up the array's device address (cudaGetSymbolAddress) with that device
 * current, and keeps it for the life of the process; after a cudaDeviceReset
 * of that device the kept address is stale, so do not call this entry point
 * on a device that was reset in the same process.  Make the first call on a
 * device before any stream capture.  All calls share
 * the one array: calls that overlap on the GPU (different streams or host
 * threads, same device) race and may return wrong sums.  Returns LBM_ESIZE if
 * the reduction would need more than the array's 1024 block records (more
 * than 256 SMs), LBM_EINVAL for null or misaligned pointers. */
int lbm_conservation_noalloc(lbm_handle h, const void *state, void *stream, double *out);

/* Sampled read-back of the current state: for `count` (<= 2^20) nodes
 * given by their indices node = x + X (y + Y z) in the device array `nodes`
 * (int64; the caller keeps them below X*Y*Z), writes all Q + Q_r populations,
 * decoded to float, to the device array out[k * (Q + Q_r) + i] (translational
 * i < Q first, then the rotational ones).  For checks of states too large to
 * copy back whole.  Asynchronous. */
int lbm_sample_state(lbm_handle h, const int64_t *nodes, int count, float *out);

/* Copy the stored populations to / from device arrays in canonical order:
 * ft[i*N + node] for i < Q_t, fr[j*N + node] for j < Q_r (fr ignored when
 * n = 0).  In STREAM mode ft holds post-collision values (the pull source).
 * Asynchronous.  Used for checkpoint/resume and per-population checks. */
int lbm_get_state(lbm_handle h, float *ft, float *fr);
int lbm_set_state(lbm_handle h, const float *ft, const float *fr);

/* Sticky device status: LBM_OK or LBM_ENONFINITE.  Synchronizing. */
int lbm_status(lbm_handle h);

/* Steps taken since the last lbm_set_macro / lbm_set_state. */
int64_t lbm_steps(lbm_handle h);

/* Human-readable message for the last error on this handle ("" if none). */
const char *lbm_last_error(lbm_handle h);

/* The library's own lattice constants (Tables I, II as re-solved here, in
 * double precision before rounding): r, e[Q*3] (ints), w[Q].  Returns Q, or
 * a negative lbm_status.  Host only; needs no GPU. */
int lbm_lattice_info(int lattice, double *r, int *e, double *w);

/* Number of kernel launches this handle has enqueued since creation. */
int64_t lbm_launch_count(lbm_handle h);

void lbm_destroy(lbm_handle h);

/* ---------------------------------------------------------------------------
 * Ensembles of independent 1-D problems in one persistent launch.
 *
 * `count` shock tubes (or any 1-D problems), each on D1Q7 + D1Q7 (Table II)
 * with copy (zero-gradient) ends, each with its own length L_k, rotational
 * degrees n_k (gamma_k = (3+n_k)/(1+n_k), Sec. III) and relaxation time
 * tau_k, all advanced by the same step as lbm_step (Sec. V; STREAM or FD
 * transport, one mode per ensemble) and giving bit-identical results to
 * running each problem through its own lbm_handle.  One launch advances every
 * problem by k steps: blocks stay resident and claim whole problems, longest
 * first, through an atomic counter; each block runs all k steps of its
 * problem with a block barrier between steps, so a problem's state stays in
 * L2 while it is worked on.  The launch (counter reset + kernel) is built
 * once as a CUDA graph and replayed.  Every problem carries 7 rotational
 * populations (with n_k = 0 they carry no energy).
 *
 * Layout.  Macro fields are float32 device arrays of total_nodes = sum L_k
 * entries, problem k at node offset sum_{j<k} L_j (u has one component).
 * The state buffers hold, for problem k, 14 arrays of roundup(L_k, 32)
 * floats.  As for lbm_handle, the caller allocates two state buffers and a
 * work buffer (per-problem table, per-problem status words, the counter) of
 * the reported sizes, 256-byte aligned; the library allocates no device
 * memory.  Status: a non-finite or non-positive rho or T in problem k sets
 * bit 0 of its status word; lbm_batch_status reads them. */
typedef struct lbm_batch_ctx *lbm_batch;

/* count >= 1; lengths[k] >= 1; n[k] >= 0; tau[k] > 0 (host arrays, copied);
 * mode LBM_MODE_STREAM or LBM_MODE_FD with m_fd >= 1 (Eq. DisEvolSpaTiI).
 * The state must stay below 2^31 floats (LBM_ESIZE otherwise). */
int lbm_batch_create(int count, const int64_t *lengths, const int *n, const double *tau,
                     int mode, int m_fd, lbm_batch *out);

/* Give the problems of an existing ensemble new rotational degree counts
 * n[count] and relaxation times tau[count] (host arrays), keeping their
 * lengths, buffers and cached launch graphs; a solver pool can so serve
 * changing sets of problems of one length.  The state is invalidated:
 * lbm_batch_set_macro must follow before lbm_batch_run. */
int lbm_batch_set_problems(lbm_batch b, const int *n, const double *tau);

/* Bytes for each state buffer and for the work buffer; total node count. */
int lbm_batch_sizes(lbm_batch b, size_t *state_bytes, size_t *work_bytes, int64_t *total_nodes);

/* Restrict, per problem, the nodes whose failure (non-finite or
 * non-positive rho or T) sets the status word to [lo[k], hi[k]) (host
 * arrays, 0 <= lo <= hi <= length); lo = hi = NULL restores whole
 * problems.  A window of a longer problem run with margins reports only
 * failures of its exact interior.  Keeps the state and the cached graphs;
 * no counterpart in the paper. */
int lbm_batch_set_watch(lbm_batch b, const int *lo, const int *hi);

/* Bind caller memory and the stream; uploads the per-problem table
 * (asynchronously, from host memory owned by the handle). */
int lbm_batch_bind(lbm_batch b, void *buf_a, void *buf_b, size_t state_bytes, void *work,
                   size_t work_bytes, void *stream);

/* Equilibrium initial state of every problem (as lbm_set_macro); clears
 * the status words.  Asynchronous. */
int lbm_batch_set_macro(lbm_batch b, const float *rho, const float *u, const float *T);

/* Advance every problem by k >= 0 steps in one persistent launch.  When
 * the longest problem has at most 864 nodes each block holds its problem's
 * two state buffers in shared memory for the whole run (same results, bit
 * for bit).  Asynchronous. */
int lbm_batch_run(lbm_batch b, int64_t k);

/* rho, u, T of every problem (layout above).  Asynchronous. */
int lbm_batch_get_moments(lbm_batch b, float *rho, float *u, float *T);

/* Per-problem status words into a HOST array of `count` ints (may be NULL)
 * and the number of problems whose word is non-zero.  Synchronizing. */
int lbm_batch_status(lbm_batch b, int *status, int *n_bad);

/* Shape of the persistent launch: threads per block (32..1024, a multiple of
 * 32) and resident blocks per SM (0 = as many as fit; fewer keep more of
 * each problem's state in L2).  lbm_batch_autotune times `sample_steps`
 * steps of the bound ensemble for every pair of 128/256/512/1024 threads and
 * 1/2/4/max blocks per SM and keeps the fastest (returned through the
 * pointers, which may be NULL).  Autotuning advances the state: call
 * lbm_batch_set_macro afterwards. */
int lbm_batch_set_block(lbm_batch b, int threads, int blocks_per_sm);
int lbm_batch_autotune(lbm_batch b, int64_t sample_steps, int *threads, int *blocks_per_sm);

int64_t lbm_batch_launch_count(lbm_batch b);
const char *lbm_batch_last_error(lbm_batch b);
void lbm_batch_destroy(lbm_batch b);

/* ------------------------------------------------------------------------
 * Learned surrogate: a 1-D convolutional operator that advances the
 * macroscopic state (rho, u, T) of a tube by K lattice steps per call.  The
 * paper has no counterpart: it is an extension of the method, which remains
 * its fallback and the reference it is measured against.  The network (all
 * entry points below are its building blocks; the layer sequence is driven
 * by the Python binding):
 *   features  a[p]     = ((rho-1)/s0, u/s1, (T-1)/s2, (gamma-1.4)/s3)
 *   lift      x0       = bf16(a Wl^T + bl)
 *   layer i   z_i      = conv(x_i; W_i, d_i) + b_i,  W_i[t][co][ci], k taps,
 *                        tap t reads position l + (t - k/2) d_i, zero outside
 *                        the tube
 *             x_{i+1}  = bf16(x_i + gelu(z_i)),  gelu in its tanh form
 *   head      out      = x_N Wp^T + bp
 *   update    (rho,u,T)' = (rho,u,T) + out * out_scale
 * Patches of P consecutive nodes may be treated as one position (F = 4P
 * features in, Fo = 3P outputs), which is a reinterpretation of the same
 * channel-last buffers.
 *
 * Common conventions.  Every pointer is a device pointer unless stated;
 * the caller owns every buffer; nothing is allocated.  Activations are
 * channel-last [B][L][C] (tube b, position l, channel c) bfloat16 with C a
 * multiple of 128, gradients of the residual stream float32 in the same
 * layout, conv weights bfloat16 [k][C][C].  `impl` selects the tensor-core
 * kernels (0: tcgen05 MMA fed by the Tensor Memory Accelerator, operands
 * 16-byte aligned, persistent blocks, 128 positions x 128 channels per
 * tile; 3: the same with 128 channels x 256 positions per tile and one
 * activation window per 64-channel chunk read by all taps, for
 * (k - 1) dil <= 64, else LBM_EINVAL; 2: one output tile per block) or the
 * CUDA-core ones (1); the weight gradient runs the same kernel for 0, 2
 * and 3.  `status` (device int, may be
 * NULL) receives bit 4 if a tensor-core kernel gave up waiting on a
 * barrier, in which case its outputs are not written.  Calls are
 * asynchronous on `stream`; they return LBM_OK, LBM_EINVAL (bad pointer,
 * shape, alignment or aliasing) or LBM_ECUDA (launch failure).
 * ---------------------------------------------------------------------- */

/* y = bf16(x + gelu(conv(x; w, dil) + bias)); z (may be NULL) receives
 * bf16(conv(x) + bias).  x, y, z: [B][L][C]; w: [k][C][C] (W[t][co][ci]);
 * bias: [C] float.  k odd, x != y. */
int lbm_nn_conv_forward(const void *x, const void *w, const float *bias, void *y, void *z, int B,
                        int L, int C, int k, int dil, int impl, int *status, void *stream);

/* Input gradient of a conv layer, added to the residual-stream gradient:
 * gx[b,l,ci] += sum_t sum_co gz[b, l - (t-k/2) dil, co] W[t][co][ci], given
 * wt = the transposed, flipped weights WT[t][ci][co] = W[k-1-t][co][ci]
 * (lbm_nn_cast_weights).  If zprev is not NULL, also the pre-activation
 * gradient of the layer below: gzprev = bf16(gx_new * gelu'(zprev)). */
int lbm_nn_conv_backward_data(const void *gz, const void *wt, float *gx, const void *zprev,
                              void *gzprev, int B, int L, int C, int k, int dil, int impl,
                              int *status, void *stream);

/* Weight gradient, accumulated: gw[t][co][ci] += sum_{b,l} gz[b,l,co] *
 * x[b, l + (t-k/2) dil, ci].  gw float [k][C][C], 16-byte aligned. */
int lbm_nn_conv_backward_weight(const void *gz, const void *x, float *gw, int B, int L, int C, int k,
                                int dil, int impl, int *status, void *stream);

/* bf16 copies of `layers` float conv weights [layers][k][C][C]: w_bf16 in
 * the same layout, wt_bf16 (may be NULL) transposed and flipped per layer. */
int lbm_nn_cast_weights(const float *w, void *w_bf16, void *wt_bf16, int layers, int C, int k,
                        void *stream);

/* Lift: x0[p][c] = bf16(sum_j feat[p][j] Wl[c][j] + bl[c]) for P positions
 * of F float features, F one of 4, 8, 16, 32 (patches of 1, 2, 4, 8 nodes),
 * feat and Wl 16-byte aligned; C a multiple of 32, at most 1024. */
int lbm_nn_lift(const float *feat, const float *Wl, const float *bl, void *x0, int64_t P, int F,
                int C, void *stream);

/* Lift backward, accumulated: gWl[c][j] += sum_p gx0[p][c] feat[p][j],
 * gbl[c] += sum_p gx0[p][c].  C a multiple of 32, at most 1024; F one of
 * 4, 8, 16, 32 (patches of 1, 2, 4, 8 nodes). */
int lbm_nn_lift_backward(const float *gx0, const float *feat, float *gWl, float *gbl, int64_t P,
                         int F, int C, void *stream);

/* Head: out[p][o] = sum_c x[p][c] Wp[o][c] + bp[o] for Fo = 3, 6, 12 or 24
 * float outputs (patches of 1, 2, 4, 8 nodes); C a multiple of 8, at most
 * 1024; x and Wp 16-byte aligned. */
int lbm_nn_head(const void *x, const float *Wp, const float *bp, float *out, int64_t P, int C, int Fo,
                void *stream);

/* Head backward: gx = gout Wp (written), gz = bf16(gx * gelu'(z)) (written;
 * z is the pre-activation of the last conv layer), gWp += gout^T x,
 * gbp += sum_p gout.  C is 128 or 256; Fo is 3, 6, 12 or 24 (patches of 1,
 * 2, 4, 8 nodes). */
int lbm_nn_head_backward(const float *gout, const void *x, const float *Wp, const void *z, float *gx,
                         void *gz, float *gWp, float *gbp, int64_t P, int C, int Fo, void *stream);

/* Bias gradient of a conv layer, accumulated: gb[c] += sum_p gz[p][c]. */
int lbm_nn_bias_grad(const void *gz, float *gb, int64_t P, int C, void *stream);

/* One Adam step (Kingma and Ba, bias-corrected, step number t >= 1) on n
 * float parameters: g += weight_decay p; m, v moment estimates updated in
 * place; p -= lr m_hat / (sqrt(v_hat) + eps). */
int lbm_nn_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                float eps, int t, float weight_decay, void *stream);

/* The Adam step with its per-step constants on the device, for training
 * steps captured in a CUDA graph: t = ++*step (device int64, the count of
 * completed steps), lr = lr_table[min(t, table_len) - 1] (device float
 * schedule), bias corrections 1/(1 - b1^t), 1/(1 - b2^t) written to hyper
 * (device float[3], scratch), then the update of lbm_nn_adam. */
int lbm_nn_adam_scheduled(float *p, const float *g, float *m, float *v, int64_t n,
                          const float *lr_table, int64_t table_len, int64_t *step, float *hyper,
                          float b1, float b2, float eps, float weight_decay, void *stream);

/* Training minibatch drawn on the device from the counter-based generator
 * SplitMix64: pair i takes h = splitmix64(seed ^ splitmix64(*step * batch +
 * i)), tube = good[(h & 0xffffffff) mod ngood], window j = (h >> 32) mod
 * windows, and writes rows_src[i] = j*tubes + tube, rows_dst[i] =
 * (j+1)*tubes + tube (rows of trajectory fields stored [windows+1][tubes][L])
 * and gamma_out[i] = gamma_tubes[tube].  good: device int[ngood] indices of
 * the usable tubes. */
int lbm_nn_sample_pairs(const int *good, int ngood, int windows, int tubes,
                        const float *gamma_tubes, uint64_t seed, const int64_t *step, int batch,
                        int64_t *rows_src, int64_t *rows_dst, float *gamma_out, void *stream);

/* Mean squared error: *loss += mean((out - target)^2) (device double, the
 * caller zeroes it); gout (may be NULL) = 2 (out - target) / n. */
int lbm_nn_mse(const float *out, const float *target, float *gout, double *loss, int64_t n,
               void *stream);

/* Features of B tubes of L nodes: feat[b*L+l] = the four values above;
 * gamma[B] per tube; in_scale: 4 HOST floats.  feat 16-byte aligned. */
int lbm_nn_features(const float *rho, const float *u, const float *T, const float *gamma, float *feat,
                    int B, int L, const float *in_scale, void *stream);

/* Training targets: target[i] = ((rho2-rho)/s0, (u2-u)/s1, (T2-T)/s2) for n
 * nodes; out_scale: 3 HOST floats. */
int lbm_nn_targets(const float *rho, const float *u, const float *T, const float *rho2,
                   const float *u2, const float *T2, float *target, int64_t n,
                   const float *out_scale, void *stream);

/* Update: (rho2, u2, T2) = (rho, u, T) + out * out_scale (HOST floats). */
int lbm_nn_apply(const float *rho, const float *u, const float *T, const float *out, float *rho2,
                 float *u2, float *T2, int64_t n, const float *out_scale, void *stream);

/* Per-tube checks over the window [w0, w0+W) of B tubes of L nodes between
 * a state (rho, u, T) and a second state (rho2, u2, T2):
 *   residual[b] (may be NULL) = max of the relative changes of the totals of
 *     mass, momentum (relative to the mass) and energy
 *     rho ((1+n)/2 T + u^2/2), half_dof[b] = (1+n)/2; +infinity if the
 *     second state has a non-positive or non-finite rho or T, or a
 *     non-finite u, anywhere in the window;
 *   l1[b] (may be NULL) = max over rho, u, T of sum|first - second| over
 *     the window divided by sum|rho2|, sum sqrt(gamma T2) and sum|T2|
 *     (the second state is the reference);
 *   starts (may be NULL; device int[2B]) = a spot-check window of `span`
 *     nodes centred on the node where |rho2 - rho| is largest (the first one
 *     on ties; a non-finite change counts as largest):
 *     starts[b] = clamp(argmax - span/2, 0, L - span), starts[B + b] =
 *     starts[b] + margin (0 <= 2 margin <= span <= L). */
int lbm_nn_tube_checks(const float *rho, const float *u, const float *T, const float *rho2,
                       const float *u2, const float *T2, const float *half_dof, const float *gamma,
                       float *residual, float *l1, int *starts, int span, int margin, int B, int L,
                       int w0, int W, void *stream);

/* Self-test of the bounded barrier wait the tensor-core kernels use (a
 * library service, no counterpart in the paper): one thread waits on a
 * shared-memory barrier that nothing completes unless `arrive` is set; after
 * budget_cycles (<= 2^34) clock cycles the wait gives up and sets bit 4 of
 * the device int *status, exactly as a stalled convolution kernel would.
 * Lets a test confirm, without faulting or hanging the GPU, that such a
 * stall ends in a status the host can read. */
int lbm_nn_wait_selftest(long long budget_cycles, int arrive, int *status, void *stream);

/* Row gather of three float fields stored as rows of row_len nodes:
 * d_f[i*W + w] = f[rows[i]*row_len + offsets[i] + w] for i < count, w < W
 * (rows: device int64, offsets: device int or NULL for 0).  Used for the
 * training minibatches, the spot-check windows and the fallback tubes; the
 * caller keeps offsets[i] + W <= row_len. */
int lbm_nn_gather(const float *a, const float *b, const float *c, const int64_t *rows,
                  const int *offsets, int count, int64_t row_len, int W, float *da, float *db,
                  float *dc, void *stream);

/* The reverse assignment: f[rows[i]*row_len + offsets[i] + w] = d_f[i*W + w]
 * (here a, b, c are the packed rows and da, db, dc the row-major fields). */
int lbm_nn_scatter(const float *a, const float *b, const float *c, const int64_t *rows,
                   const int *offsets, int count, int64_t row_len, int W, float *da, float *db,
                   float *dc, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
