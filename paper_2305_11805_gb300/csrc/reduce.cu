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

// one warp per configuration: lane l sums the chunks l, l + 32, ... in order, then a fixed
// butterfly joins the lanes (the same order on every call: energies are bit-reproducible)
__global__ void __launch_bounds__(kCfgRedWarps * 32)
k_cfg_final(int64_t C, int B, const double* __restrict__ part, double* __restrict__ E_cfg,
            double* __restrict__ virial)
{
    const int lane = threadIdx.x & 31;
    const int64_t c = (int64_t)blockIdx.x * kCfgRedWarps + (threadIdx.x >> 5);
    if (c >= C) return;
    double v[kCfgVals];
#pragma unroll
    for (int k = 0; k < kCfgVals; ++k) v[k] = 0.0;
    for (int b = lane; b < B; b += 32)
#pragma unroll
        for (int k = 0; k < kCfgVals; ++k) v[k] += part[((size_t)c * B + b) * kCfgVals + k];
#pragma unroll
    for (int k = 0; k < kCfgVals; ++k)
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if (lane == 0 && E_cfg) E_cfg[c] = v[0];
    if (lane == 0 && virial)
#pragma unroll
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
    k_cfg_final<<<(unsigned)((w.C + kCfgRedWarps - 1) / kCfgRedWarps), kCfgRedWarps * 32, 0, s>>>(w.C, B, part,
                                                                                                  E_cfg, virial);
    *launches += 2;
    return cudaGetLastError();
}

// ------------------------------------------------------------------ loss

constexpr int kLossBlocks = 120;

// loss term and its slope: kind 0 = x^2, 1 = exp(x^2) - 1
__device__ __forceinline__ double loss_term(int kind, double x) { return kind ? expm1(x * x) : x * x; }
__device__ __forceinline__ double loss_slope(int kind, double x) { return kind ? 2.0 * x * exp(x * x) : 2.0 * x; }

// C_norm and N_norm are the loss normalisers: the batch's own counts, or the global counts
// of a data-parallel batch split over ranks.  Energy differences per configuration or, with
// e_per_atom, divided by the configuration's atom count.
__global__ void k_loss_partial(int64_t C, int64_t N, double C_norm, double N_norm, LossOpts lo,
                               const int64_t* __restrict__ atom_off, const double* __restrict__ E_cfg,
                               const double* __restrict__ E_ref, const float* __restrict__ F,
                               const float* __restrict__ F_ref, double w_force, double* __restrict__ part,
                               double* __restrict__ alpha_cfg, float* __restrict__ u)
{
    double le = 0.0, lf = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double cu = w_force / (3.0 * N_norm);
    for (int64_t c = t0; c < C; c += stride) {
        const int64_t n = atom_off[c + 1] - atom_off[c];
        const double per = (lo.e_per_atom && n > 0) ? 1.0 / (double)n : 1.0;
        const double d = (E_cfg[c] - E_ref[c]) * per;
        le += loss_term(lo.e_kind, d);
        alpha_cfg[c] = loss_slope(lo.e_kind, d) * per / C_norm;
    }
    for (int64_t k = t0; k < 3 * N; k += stride) {
        const double r = (double)F[k] - (double)F_ref[k];
        lf += loss_term(lo.f_kind, r);
        u[k] = (float)(cu * loss_slope(lo.f_kind, r));
    }
    double a = block_sum_d(le);
    double b = block_sum_d(lf);
    if (threadIdx.x == 0) { part[2 * blockIdx.x] = a; part[2 * blockIdx.x + 1] = b; }
}

// sums of |w| and w^2 over the weights in wr (same grid as k_loss_partial)
__global__ void k_penalty_partial(ParamRanges wr, const float* __restrict__ theta, double* __restrict__ part)
{
    double s1 = 0.0, s2 = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int q = 0; q < wr.n; ++q)
        for (int64_t k = t0; k < wr.len[q]; k += stride) {
            const double w = theta[wr.off[q] + k];
            s1 += fabs(w);
            s2 += w * w;
        }
    double a = block_sum_d(s1);
    double b = block_sum_d(s2);
    if (threadIdx.x == 0) { part[2 * blockIdx.x] = a; part[2 * blockIdx.x + 1] = b; }
}

__global__ void k_loss_final(double C_norm, double N_norm, double w_force, LossOpts lo, int penalty,
                             const double* __restrict__ part, double* __restrict__ loss)
{
    const int lane = threadIdx.x & 31;
    double le = 0.0, lf = 0.0, l1 = 0.0, l2 = 0.0;
    for (int b = lane; b < kLossBlocks; b += 32) {
        le += part[2 * b];
        lf += part[2 * b + 1];
        if (penalty) { l1 += part[2 * kLossBlocks + 2 * b]; l2 += part[2 * kLossBlocks + 2 * b + 1]; }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        le += __shfl_xor_sync(0xffffffffu, le, o);
        lf += __shfl_xor_sync(0xffffffffu, lf, o);
        l1 += __shfl_xor_sync(0xffffffffu, l1, o);
        l2 += __shfl_xor_sync(0xffffffffu, l2, o);
    }
    if (lane == 0 && blockIdx.x == 0) *loss = le / C_norm + w_force * lf / (3.0 * N_norm) + lo.l1 * l1 + lo.l2 * l2;
}

cudaError_t launch_loss(const Work& w, int64_t C_norm, int64_t N_norm, const LossOpts& lo, const ParamRanges& wr,
                        const float* theta, const double* E_cfg, const double* E_ref, const float* F,
                        const float* F_ref, double w_force, double* loss, double* alpha_cfg, float* u, double* part,
                        cudaStream_t s, int* launches)
{
    const double cn = (double)(C_norm > 0 ? C_norm : w.C), nn = (double)(N_norm > 0 ? N_norm : w.N);
    k_loss_partial<<<kLossBlocks, kRedThreads, 0, s>>>(w.C, w.N, cn, nn, lo, w.sys->atom_off, E_cfg, E_ref, F, F_ref,
                                                       w_force, part, alpha_cfg, u);
    const int penalty = (lo.l1 != 0.0 || lo.l2 != 0.0) ? 1 : 0;
    if (penalty) {
        k_penalty_partial<<<kLossBlocks, kRedThreads, 0, s>>>(wr, theta, part + 2 * kLossBlocks);
        ++*launches;
    }
    k_loss_final<<<1, 32, 0, s>>>(cn, nn, w_force, lo, penalty, part, loss);
    *launches += 2;
    return cudaGetLastError();
}

__global__ void k_penalty_grad(ParamRanges wr, double l1, double l2, const float* __restrict__ theta,
                               float* __restrict__ dtheta)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int q = 0; q < wr.n; ++q)
        for (int64_t k = t0; k < wr.len[q]; k += stride) {
            const int64_t i = wr.off[q] + k;
            const float w = theta[i];
            dtheta[i] += (float)(l1 * (double)((w > 0.f) - (w < 0.f)) + 2.0 * l2 * (double)w);
        }
}

cudaError_t launch_penalty_grad(const LossOpts& lo, const ParamRanges& wr, const float* theta, float* dtheta,
                                cudaStream_t s, int* launches)
{
    if (lo.l1 == 0.0 && lo.l2 == 0.0) return cudaSuccess;
    k_penalty_grad<<<kLossBlocks, kRedThreads, 0, s>>>(wr, lo.l1, lo.l2, theta, dtheta);
    ++*launches;
    return cudaGetLastError();
}

// ------------------------------------------------------------------ Adam

// One Adam step (Kingma and Ba, Algorithm 1) fused in one pass: m = b1 m + (1 - b1) g,
// v = b2 v + (1 - b2) g^2, theta -= lr (m / c1) / (sqrt(v / c2) + eps) with the bias
// corrections c1 = 1 - b1^t, c2 = 1 - b2^t; entries inside a frozen range are skipped.
__global__ void k_adam(int64_t P, float* __restrict__ theta, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float c1, float c2, float eps,
                       ParamRanges frozen)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P) return;
    for (int q = 0; q < frozen.n; ++q)
        if (k >= frozen.off[q] && k < frozen.off[q] + frozen.len[q]) return;
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.f - b1) * gk;
    const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    theta[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

cudaError_t launch_adam(int64_t P, float* theta, const float* g, float* m, float* v, double lr, double b1, double b2,
                        double c1, double c2, double eps, const ParamRanges& frozen, cudaStream_t s, int* launches)
{
    if (P == 0) return cudaSuccess;
    k_adam<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(P, theta, g, m, v, (float)lr, (float)b1, (float)b2, (float)c1,
                                                       (float)c2, (float)eps, frozen);
    ++*launches;
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
