// FP64 reductions: per-configuration energies and virials (sum of atomic energies,
// Sec. II), and the energy + force training loss (Sec. II.A) with its seeds for the
// reverse pass.  Every reduction runs in a fixed order, so results are deterministic.
#include "common.cuh"

namespace panna {

constexpr int kRedThreads = 256;
constexpr int kCfgVals = 10;   // energy + 9 virial entries

__device__ __forceinline__ double block_sum_d(double v)
{
    __shared__ double sh[kRedThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < kRedThreads / 32; ++k) t += sh[k];
    return t;   // valid in thread 0
}

// partial sums over chunk b of configuration c: one warp per (configuration, chunk)
constexpr int kCfgRedWarps = 8;

__global__ void __launch_bounds__(kCfgRedWarps * 32)
k_cfg_partial(int64_t C, const int64_t* __restrict__ atom_off, int B, const int32_t* __restrict__ row_of_atom,
              const float* __restrict__ E_rows, const float* __restrict__ vir_atom, float* __restrict__ E_atom,
              double* __restrict__ part)
{
    const int lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * kCfgRedWarps + (threadIdx.x >> 5);
    if (gw >= C * B) return;
    const int64_t c = gw / B;
    const int b = (int)(gw % B);
    const int64_t a0 = atom_off[c], a1 = atom_off[c + 1];
    const int64_t per = (a1 - a0 + B - 1) / B;
    const int64_t s0 = a0 + b * per, s1 = min(a1, s0 + per);
    double v[kCfgVals];
#pragma unroll
    for (int k = 0; k < kCfgVals; ++k) v[k] = 0.0;
    for (int64_t i = s0 + lane; i < s1; i += 32) {
        const int row = row_of_atom[i];
        const float e = row >= 0 ? E_rows[row] : 0.f;     // a ghost (row -1) adds nothing
        if (E_atom) E_atom[i] = e;
        if (row < 0) continue;
        v[0] += e;
        if (vir_atom)
#pragma unroll
            for (int k = 0; k < 9; ++k) v[1 + k] += vir_atom[9 * i + k];
    }
#pragma unroll
    for (int k = 0; k < kCfgVals; ++k)
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if (lane == 0) {
        double* out = part + ((size_t)c * B + b) * kCfgVals;
#pragma unroll
        for (int k = 0; k < kCfgVals; ++k) out[k] = v[k];
    }
}

__global__ void k_cfg_final(int64_t C, int B, const double* __restrict__ part, double* __restrict__ E_cfg,
                            double* __restrict__ virial)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    double v[kCfgVals];
    for (int k = 0; k < kCfgVals; ++k) v[k] = 0.0;
    for (int b = 0; b < B; ++b)
        for (int k = 0; k < kCfgVals; ++k) v[k] += part[((size_t)c * B + b) * kCfgVals + k];
    if (E_cfg) E_cfg[c] = v[0];
    if (virial)
        for (int k = 0; k < 9; ++k) virial[9 * c + k] = v[1 + k];
}

int cfg_chunks(int64_t N, int64_t C)
{
    int64_t B = N / (C * 256) + 1;
    return (int)(B > 8192 ? 8192 : B);
}

cudaError_t launch_cfg_reduce(const Work& w, const float* E_rows, const float* vir_atom, double* E_cfg, double* virial,
                              float* E_atom, double* part, cudaStream_t s, int* launches)
{
    const int B = cfg_chunks(w.N, w.C);
    k_cfg_partial<<<(unsigned)((w.C * B + kCfgRedWarps - 1) / kCfgRedWarps), kCfgRedWarps * 32, 0, s>>>(
        w.C, w.sys->atom_off, B, w.row_of_atom, E_rows, vir_atom, E_atom, part);
    k_cfg_final<<<(unsigned)((w.C + 127) / 128), 128, 0, s>>>(w.C, B, part, E_cfg, virial);
    *launches += 2;
    return cudaGetLastError();
}

// ------------------------------------------------------------------ loss

constexpr int kLossBlocks = 120;

// C_norm and N_norm are the loss normalisers: the batch's own counts, or the global counts
// of a data-parallel batch split over ranks
__global__ void k_loss_partial(int64_t C, int64_t N, double C_norm, double N_norm, const double* __restrict__ E_cfg,
                               const double* __restrict__ E_ref, const float* __restrict__ F,
                               const float* __restrict__ F_ref, double w_force, double* __restrict__ part,
                               double* __restrict__ alpha_cfg, float* __restrict__ u)
{
    double le = 0.0, lf = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double cu = 2.0 * w_force / (3.0 * N_norm);
    for (int64_t c = t0; c < C; c += stride) {
        double r = E_cfg[c] - E_ref[c];
        le += r * r;
        alpha_cfg[c] = 2.0 * r / C_norm;
    }
    for (int64_t k = t0; k < 3 * N; k += stride) {
        double r = (double)F[k] - (double)F_ref[k];
        lf += r * r;
        u[k] = (float)(cu * r);
    }
    double a = block_sum_d(le);
    double b = block_sum_d(lf);
    if (threadIdx.x == 0) { part[2 * blockIdx.x] = a; part[2 * blockIdx.x + 1] = b; }
}

__global__ void k_loss_final(double C_norm, double N_norm, double w_force, const double* __restrict__ part,
                             double* __restrict__ loss)
{
    const int lane = threadIdx.x & 31;
    double le = 0.0, lf = 0.0;
    for (int b = lane; b < kLossBlocks; b += 32) { le += part[2 * b]; lf += part[2 * b + 1]; }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        le += __shfl_xor_sync(0xffffffffu, le, o);
        lf += __shfl_xor_sync(0xffffffffu, lf, o);
    }
    if (lane == 0 && blockIdx.x == 0) *loss = le / C_norm + w_force * lf / (3.0 * N_norm);
}

cudaError_t launch_loss(const Work& w, int64_t C_norm, int64_t N_norm, const double* E_cfg, const double* E_ref,
                        const float* F, const float* F_ref, double w_force, double* loss, double* alpha_cfg, float* u,
                        double* part, cudaStream_t s, int* launches)
{
    const double cn = (double)(C_norm > 0 ? C_norm : w.C), nn = (double)(N_norm > 0 ? N_norm : w.N);
    k_loss_partial<<<kLossBlocks, kRedThreads, 0, s>>>(w.C, w.N, cn, nn, E_cfg, E_ref, F, F_ref, w_force, part,
                                                       alpha_cfg, u);
    k_loss_final<<<1, 32, 0, s>>>(cn, nn, w_force, part, loss);
    *launches += 2;
    return cudaGetLastError();
}

// upstream gradients given directly (vector-Jacobian product): alpha_cfg = dE, u = dF
__global__ void k_alpha_rows(int64_t N, const int32_t* __restrict__ atom_cfg, const int32_t* __restrict__ row_of_atom,
                             const double* __restrict__ alpha_cfg, float* __restrict__ alpha_rows)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N || row_of_atom[i] < 0) return;
    alpha_rows[row_of_atom[i]] = alpha_cfg ? (float)alpha_cfg[atom_cfg[i]] : 0.f;
}

cudaError_t launch_row_scale(const Work& w, const double* alpha_cfg, float* alpha_rows, cudaStream_t s, int* launches)
{
    k_alpha_rows<<<(unsigned)((w.N + 255) / 256), 256, 0, s>>>(w.N, w.atom_cfg, w.row_of_atom, alpha_cfg, alpha_rows);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace panna
