// Internal interface between the host API (lbm_api.cu) and the per-lattice
// kernel translation units (lbm_<lattice>.cu).  Not part of the C ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace lbm {

constexpr int kMaxQ = 343;       // largest translational set built here (D3Q343)
constexpr int kRedThreads = 256; // threads per block of the conservation reduction
constexpr int kRedSlots = 8;     // doubles per reduction partial
constexpr int kMaxRedBlocks = 1024;

// Work-buffer layout (bytes from the start of the caller's work buffer).
constexpr size_t kWorkStatus = 0;      // int: sticky status bits
constexpr size_t kWorkResult = 256;    // kRedSlots doubles: finished reduction
constexpr size_t kWorkPartials = 512;  // kMaxRedBlocks * kRedSlots doubles
constexpr size_t kWorkBytes = kWorkPartials + sizeof(double) * kRedSlots * kMaxRedBlocks;

enum class Op { Step, Init, Moments, Conserve, GetState, SetState, Sample };

// Everything a kernel launch needs; filled by the host API.
struct Args {
    int lattice, D, Q, Qr, mode, m_fd;
    int storage;  // lbm_storage: 0 float, 1 half / 2 bfloat16 deviations from rest,
                  // 3 half / 4 bfloat16 deviations from a per-node reference
    size_t ref_offset;  // storage 3, 4: bytes from a state buffer's start to its
                        // per-node reference records (float4 per node, S of them)
    int X, Y, Z, pitch;
    int64_t S;  // population stride in floats (pitch * Y * Z)
    int64_t N;  // nodes (X * Y * Z)
    int bc[3];
    float r, omega, nu_scale, cT, half_n, half_n_r2, inv_m;
    float w[kMaxQ];
    float wr[7];
    const void *src;  // current state (Step reads, Moments/Conserve/GetState read)
    void *dst;        // next state (Step writes, Init/SetState write)
    const float *in0, *in1, *in2;  // Init: rho, u, T; SetState: ft, fr
    float *out0, *out1, *out2;     // Moments: rho, u, T; GetState: ft, fr
    int *status;
    double *partials;
    int red_blocks;
    const int64_t *nodes;  // Sample: node indices (x fastest), `count` of them
    int count;
};

cudaError_t launch_d1q7(Op op, const Args &a, cudaStream_t s);
cudaError_t launch_d2q37(Op op, const Args &a, cudaStream_t s);
cudaError_t launch_d2q49(Op op, const Args &a, cudaStream_t s);
cudaError_t launch_d3q343(Op op, const Args &a, cudaStream_t s);

}  // namespace lbm
