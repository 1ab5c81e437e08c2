// Per-species multilayer perceptrons (Eq. 1) on species-sorted atom rows, FP32 CUDA-core
// path: grouped GEMMs with fused bias / activation epilogues, the input gradient
// dE/dG, the forward tangent along a descriptor direction, and the weight gradient of
// the reverse pass over forward + tangent (the double backward of the force loss).
//
// Rows of species s are seg_off[s]..seg_off[s+1]-1 (device); the tile table maps a
// CTA to (species, 128-row tile) without the host knowing the species counts, so one
// launch covers all species and the launch shape depends only on N and S.
#include <algorithm>

#include "mlp.cuh"

namespace panna {

__device__ __forceinline__ float act_f(int t, float z)
{
    switch (t) {
    case PANNA_ACT_GAUSSIAN: return __expf(-z * z);
    case PANNA_ACT_RELU: return z > 0.f ? z : 0.f;
    case PANNA_ACT_TANH: return tanhf(z);
    default: return z;
    }
}
__device__ __forceinline__ float act_d1(int t, float z)
{
    switch (t) {
    case PANNA_ACT_GAUSSIAN: return -2.f * z * __expf(-z * z);
    case PANNA_ACT_RELU: return z > 0.f ? 1.f : 0.f;
    case PANNA_ACT_TANH: { float h = tanhf(z); return 1.f - h * h; }
    default: return 1.f;
    }
}
__device__ __forceinline__ float act_d2(int t, float z)
{
    switch (t) {
    case PANNA_ACT_GAUSSIAN: return (4.f * z * z - 2.f) * __expf(-z * z);
    case PANNA_ACT_TANH: { float h = tanhf(z); return -2.f * h * (1.f - h * h); }
    default: return 0.f;
    }
}

__global__ void k_tiles(int S, const int32_t* __restrict__ seg_off, int32_t* __restrict__ tile_start)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int t = 0;
        for (int s = 0; s < S; ++s) {
            tile_start[s] = t;
            t += (seg_off[s + 1] - seg_off[s] + kGM - 1) / kGM;
        }
        tile_start[S] = t;
    }
}

__device__ __forceinline__ bool tile_species(int S, const int32_t* tile_start, int tile, int& s)
{
    if (tile >= tile_start[S]) return false;
    s = 0;
    while (tile >= tile_start[s + 1]) ++s;
    return true;
}

// C[rows, N] = op(A)[rows, K] * op(B)[K, N]
//   B_TRANS (forward / tangent): op(B)[k][n] = W[n*K + k] (W is [N, K])
//   else     (input gradient):   op(B)[k][n] = W[k*N + n] (W is [K, N])
// PRO_DACT: A[r][k] is multiplied by act'(Zp[r][k]) on load (layer activation la.pact).
// EPI_FWD:  C = Z = acc + b, C2 = act(Z);  EPI_TAN: C = acc, C2 = act'(Ze) * acc.
//
// BM x 128 tile per CTA of 256 threads, BM = 128 or 64; each thread owns BM/16 x 8 outputs
// (rows ty*4 + {0..3}, and 64 + ty*4 + {0..3} when BM = 128; columns tx*4 + {0..3} and
// 64 + tx*4 + {0..3}), so its shared-memory reads are float4 and conflict-free.  K advances 8
// at a time through double-buffered shared tiles; the next tile's global loads are issued
// before the current tile's FMAs.  Every output is one FMA chain in k order, as in a plain
// dot product, whatever BM.  The 64-row form splits each 128-row tile of the tile table in
// two (CTA x -> tile x/2, half x%2) and serves grids that would leave SMs with one CTA.
struct GemmLoad { float a[4], b[4]; };

template <bool B_TRANS, int PRO, int BM>
__device__ __forceinline__ void gemm_fetch(const LayerArgs& la, int s, const float* __restrict__ A, int lda,
                                           const float* __restrict__ Zp, int ldp, const float* __restrict__ W,
                                           int K, int N, int r0, int rend, int n0, int k0, int tid, GemmLoad& g)
{
    if (BM == 64) {   // A tile: 64 rows x 8 k; thread -> row tid/4, k pair (tid&3)*2
        const int r = r0 + (tid >> 2), kq = k0 + (tid & 3) * 2;
        const bool vec = ((reinterpret_cast<uintptr_t>(A) & 7) == 0) && (lda & 1) == 0;
        if (vec && r < rend && kq + 1 < K) {
            const float2 v = *reinterpret_cast<const float2*>(A + (size_t)r * lda + kq);
            g.a[0] = v.x; g.a[1] = v.y;
        } else {
#pragma unroll
            for (int j = 0; j < 2; ++j) g.a[j] = (r < rend && kq + j < K) ? A[(size_t)r * lda + kq + j] : 0.f;
        }
        if (PRO == PRO_DACT && r < rend) {
#pragma unroll
            for (int j = 0; j < 2; ++j)
                if (kq + j < K) g.a[j] *= act_d1(la.pact[s], Zp[(size_t)r * ldp + kq + j]);
        }
    } else {   // A tile: 128 rows x 8 k; thread -> row tid/2, k quad (tid&1)*4
        const int r = r0 + (tid >> 1), kq = k0 + (tid & 1) * 4;
        const bool vec = ((reinterpret_cast<uintptr_t>(A) & 15) == 0) && (lda & 3) == 0;
        if (vec && r < rend && kq + 3 < K) {
            const float4 v = *reinterpret_cast<const float4*>(A + (size_t)r * lda + kq);
            g.a[0] = v.x; g.a[1] = v.y; g.a[2] = v.z; g.a[3] = v.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) g.a[j] = (r < rend && kq + j < K) ? A[(size_t)r * lda + kq + j] : 0.f;
        }
        if (PRO == PRO_DACT && r < rend) {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (kq + j < K) g.a[j] *= act_d1(la.pact[s], Zp[(size_t)r * ldp + kq + j]);
        }
    }
    if (B_TRANS) {   // W [N, K]: 128 n x 8 k; thread -> n tid/2, k quad (tid&1)*4
        const int n = n0 + (tid >> 1), kq = k0 + (tid & 1) * 4;
        // per-species weights start anywhere in theta: vector loads only from a 16-byte aligned base
        const bool vec = ((reinterpret_cast<uintptr_t>(W) & 15) == 0) && (K & 3) == 0;
        if (vec && n < N && kq + 3 < K) {
            const float4 v = *reinterpret_cast<const float4*>(W + (size_t)n * K + kq);
            g.b[0] = v.x; g.b[1] = v.y; g.b[2] = v.z; g.b[3] = v.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) g.b[j] = (n < N && kq + j < K) ? W[(size_t)n * K + kq + j] : 0.f;
        }
    } else {         // W [K, N]: 8 k x 128 n; thread -> k tid/32, n quad (tid&31)*4
        const int k = k0 + (tid >> 5), nq = n0 + (tid & 31) * 4;
        const bool vec = ((reinterpret_cast<uintptr_t>(W) & 15) == 0) && (N & 3) == 0;
        if (vec && k < K && nq + 3 < N) {
            const float4 v = *reinterpret_cast<const float4*>(W + (size_t)k * N + nq);
            g.b[0] = v.x; g.b[1] = v.y; g.b[2] = v.z; g.b[3] = v.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) g.b[j] = (k < K && nq + j < N) ? W[(size_t)k * N + nq + j] : 0.f;
        }
    }
}

template <bool B_TRANS, int BM>
__device__ __forceinline__ void gemm_stash(const GemmLoad& g, float (*As)[kGM], float (*Bs)[kGN], int tid)
{
    if (BM == 64) {
        const int m = tid >> 2, kq = (tid & 3) * 2;
#pragma unroll
        for (int j = 0; j < 2; ++j) As[kq + j][m] = g.a[j];
    } else {
        const int m = tid >> 1, kq = (tid & 1) * 4;
#pragma unroll
        for (int j = 0; j < 4; ++j) As[kq + j][m] = g.a[j];
    }
    if (B_TRANS) {   // 128 n x 8 k: n tid/2, k quad (tid&1)*4
        const int n = tid >> 1, kq = (tid & 1) * 4;
#pragma unroll
        for (int j = 0; j < 4; ++j) Bs[kq + j][n] = g.b[j];
    } else {
        *reinterpret_cast<float4*>(&Bs[tid >> 5][(tid & 31) * 4]) = make_float4(g.b[0], g.b[1], g.b[2], g.b[3]);
    }
}

template <bool B_TRANS, int PRO, int EPI, int BM>
__global__ void __launch_bounds__(256, 2)
k_gemm(LayerArgs la, const float* __restrict__ theta, const int32_t* __restrict__ seg_off,
       const int32_t* __restrict__ tile_start, const float* __restrict__ A, int lda,
       const float* __restrict__ Zp, int ldp, float* __restrict__ C, int ldc, float* __restrict__ C2,
       const float* __restrict__ Ze, int lde)
{
    __shared__ __align__(16) float As[2][kGK][kGM];
    __shared__ __align__(16) float Bs[2][kGK][kGN];
    constexpr int P = BM / 16;   // output rows per thread
    const int tile = BM == 128 ? (int)blockIdx.x : (int)(blockIdx.x >> 1);
    int s;
    if (!tile_species(la.S, tile_start, tile, s)) return;
    const int K = la.K[s], N = la.N[s];
    const int n0 = blockIdx.y * kGN;
    if (n0 >= N) return;
    const int r0 = seg_off[s] + (tile - tile_start[s]) * kGM + (BM == 128 ? 0 : (int)(blockIdx.x & 1) * 64);
    const int rend = seg_off[s + 1];
    if (r0 >= rend) return;   // second half of a species' last tile
    const float* W = theta + la.w_off[s];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    float acc[P][8];
#pragma unroll
    for (int a = 0; a < P; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
    GemmLoad g;
    gemm_fetch<B_TRANS, PRO, BM>(la, s, A, lda, Zp, ldp, W, K, N, r0, rend, n0, 0, tid, g);
    gemm_stash<B_TRANS, BM>(g, As[0], Bs[0], tid);
    __syncthreads();
    const int nk = (K + kGK - 1) / kGK;
    for (int t = 0; t < nk; ++t) {
        const int cur = t & 1;
        if (t + 1 < nk)
            gemm_fetch<B_TRANS, PRO, BM>(la, s, A, lda, Zp, ldp, W, K, N, r0, rend, n0, (t + 1) * kGK, tid, g);
#pragma unroll
        for (int kk = 0; kk < kGK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][kk][ty * 4]);
            const float4 a1 = BM == 128 ? *reinterpret_cast<const float4*>(&As[cur][kk][64 + ty * 4]) : a0;
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[cur][kk][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[cur][kk][64 + tx * 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int p = 0; p < P; ++p)
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[p][q] = fmaf(a[p], b[q], acc[p][q]);
        }
        if (t + 1 < nk) gemm_stash<B_TRANS, BM>(g, As[cur ^ 1], Bs[cur ^ 1], tid);
        __syncthreads();
    }
    // epilogue: each thread's 4 consecutive columns go out as one float4 where the row start
    // is 16-byte aligned, so a warp writes whole 256-byte row segments
    const float* bias = theta + la.b_off[s];
    const bool vst = ((reinterpret_cast<uintptr_t>(C) & 15) == 0) && (ldc & 3) == 0 &&
                     (EPI == EPI_STORE || ((reinterpret_cast<uintptr_t>(C2) & 15) == 0));
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int r = r0 + (p < 4 ? ty * 4 + p : 64 + ty * 4 + p - 4);
        if (r >= rend) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int nb = n0 + h * 64 + tx * 4;
            float v[4], v2[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int n = nb + j;
                v[j] = acc[p][h * 4 + j];
                v2[j] = 0.f;
                if (n >= N) continue;
                if (EPI == EPI_FWD) {
                    v[j] += bias[n];
                    v2[j] = act_f(la.act[s], v[j]);
                } else if (EPI == EPI_TAN) {
                    v2[j] = act_d1(la.act[s], Ze[(size_t)r * lde + n]) * v[j];
                }
            }
            float* c = C + (size_t)r * ldc + nb;
            float* c2 = EPI == EPI_STORE ? nullptr : C2 + (size_t)r * ldc + nb;
            if (vst && nb + 3 < N) {
                *reinterpret_cast<float4*>(c) = make_float4(v[0], v[1], v[2], v[3]);
                if (EPI != EPI_STORE) *reinterpret_cast<float4*>(c2) = make_float4(v2[0], v2[1], v2[2], v2[3]);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (nb + j >= N) break;
                    c[j] = v[j];
                    if (EPI != EPI_STORE) c2[j] = v2[j];
                }
            }
        }
    }
}

// part[split][w_off + m*K + n] = sum over rows of Zb[r][m] * A[r][n] (+ Zdb[r][m] * Ad[r][n]);
// column n == K is the bias (A = 1, Ad = 0) -> part[split][b_off + m].
// la.K = input width (n), la.N = output width (m).
__global__ void __launch_bounds__(256)
k_wgrad(LayerArgs la, const int32_t* __restrict__ seg_off, int splits,
        const float* __restrict__ Zb, const float* __restrict__ A, int ldz, int lda,
        const float* __restrict__ Zdb, const float* __restrict__ Ad, float* __restrict__ part, int64_t P)
{
    __shared__ float As[kBK][kBM + 4];
    __shared__ float Bs[kBK][kBN + 4];
    const int s = blockIdx.z / splits, split = blockIdx.z % splits;
    const int K = la.K[s], N = la.N[s];
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * kBN;
    if (m0 >= N || n0 >= K + 1) return;
    const int rs = seg_off[s], re = seg_off[s + 1];
    const int cnt = re - rs;
    const int per = (cnt + splits - 1) / splits;
    const int r0 = rs + split * per;
    const int r1 = min(re, r0 + per);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    const int npass = Zdb ? 2 : 1;
    for (int pass = 0; pass < npass; ++pass) {
        const float* Zs = pass ? Zdb : Zb;
        const float* As_src = pass ? Ad : A;
        const float one = pass ? 0.f : 1.f;
        for (int k0 = r0; k0 < r1; k0 += kBK) {
            {
                const int kk = tid >> 4, q4 = (tid & 15) * 4;
                const int r = k0 + kk;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int m = m0 + q4 + j, n = n0 + q4 + j;
                    As[kk][q4 + j] = (r < r1 && m < N) ? Zs[(size_t)r * ldz + m] : 0.f;
                    float bv = 0.f;
                    if (r < r1) {
                        if (n < K) bv = As_src[(size_t)r * lda + n];
                        else if (n == K) bv = one;
                    }
                    Bs[kk][q4 + j] = bv;
                }
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < kBK; ++kk) {
                float a[4], b[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) { a[q] = As[kk][ty * 4 + q]; b[q] = Bs[kk][tx * 4 + q]; }
#pragma unroll
                for (int p = 0; p < 4; ++p)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(a[p], b[q], acc[p][q]);
            }
            __syncthreads();
        }
    }
    float* out = part + (size_t)split * P;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int m = m0 + ty * 4 + p;
        if (m >= N) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int n = n0 + tx * 4 + q;
            if (n < K) out[la.w_off[s] + (size_t)m * K + n] = acc[p][q];
            else if (n == K) out[la.b_off[s] + m] = acc[p][q];
        }
    }
}

__global__ void k_reduce_splits(int64_t P, int splits, const float* __restrict__ part, float* __restrict__ out)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    float s = 0.f;
    for (int k = 0; k < splits; ++k) s += part[(size_t)k * P + p];
    out[p] = s;
}

// Reverse-pass seeds and elementwise adjoints of one layer:
//   Zb  = Ab * act'(Z) + Adb * act''(Z) * Zd,   Zdb = Adb * act'(Z)
__global__ void k_layer_adjoint(LayerArgs la, const int32_t* __restrict__ seg_off, int64_t N, int ld,
                                const float* __restrict__ Ab, const float* __restrict__ Adb,
                                const float* __restrict__ Z, const float* __restrict__ Zd,
                                float* __restrict__ Zb, float* __restrict__ Zdb)
{
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * ld) return;
    const int64_t r = idx / ld;
    const int c = (int)(idx % ld);
    if (r >= seg_off[la.S]) return;     // rows past the last species (ghost atoms have none)
    int s = 0;
    while (s < la.S - 1 && r >= seg_off[s + 1]) ++s;
    if (c >= la.N[s]) return;
    const int t = la.act[s];
    const float z = Z[idx];
    const float d1 = act_d1(t, z);
    Zb[idx] = Ab[idx] * d1 + Adb[idx] * act_d2(t, z) * Zd[idx];
    Zdb[idx] = Adb[idx] * d1;
}

// last-layer seeds: Ab = alpha_row (energy part), Adb = -1 (force part), widths 1
__global__ void k_seed(int64_t N, int ld, const float* __restrict__ alpha_rows, float beta,
                       float* __restrict__ Ab, float* __restrict__ Adb)
{
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    Ab[r * ld] = alpha_rows ? alpha_rows[r] : 1.f;
    if (Adb) Adb[r * ld] = beta;
}

// ----------------------------------------------------------------------------- host side

static LayerArgs layer_args(const MlpPlan& p, int l, bool backward)
{
    LayerArgs la{};
    la.S = p.S;
    for (int s = 0; s < p.S; ++s) {
        const int in = p.widths[s][l], out = p.widths[s][l + 1];
        la.K[s] = backward ? out : in;
        la.N[s] = backward ? in : out;
        la.act[s] = p.acts[s][l];
        la.pact[s] = p.acts[s][l];
        la.w_off[s] = p.w_off[s][l];
        la.b_off[s] = p.b_off[s][l];
    }
    return la;
}

static dim3 gemm_grid(const MlpPlan& p, int64_t N, int n_max)
{
    return dim3((unsigned)((N + kGM - 1) / kGM + p.S), (unsigned)((n_max + kGN - 1) / kGN), 1);
}

static int device_sms()
{
    static int n_sm = 0;
    if (n_sm == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            n_sm = v;
        else
            return 1;
    }
    return n_sm;
}

// One layer GEMM: the 64-row form (twice the CTAs, twice the resident warps per SM) when the
// 128-row grid leaves SMs with fewer than two CTAs and the reduction is short (K <= 256);
// else 128-row tiles.  On 17,780 rows the 64-row form took the K = 128 layers from 12.3 to
// 10.1 us but the K = 768 first layer from 109 to 145 us (more weight-tile traffic and fewer
// FMAs per shared-memory load), so long reductions keep the 128-row tiles.
template <bool B_TRANS, int PRO, int EPI>
static void launch_gemm(const MlpPlan& p, int64_t N, int n_max, cudaStream_t s, const LayerArgs& la,
                        const float* theta, const int32_t* seg_off, const int32_t* tile_start, const float* A,
                        int lda, const float* Zp, int ldp, float* C, int ldc, float* C2, const float* Ze, int lde)
{
    dim3 g = gemm_grid(p, N, n_max);
    int kmax = 0;
    for (int q = 0; q < la.S; ++q) kmax = std::max(kmax, la.K[q]);
    if ((int64_t)g.x * g.y < 2 * (int64_t)device_sms() && kmax <= 256) {
        g.x *= 2;
        k_gemm<B_TRANS, PRO, EPI, 64><<<g, 256, 0, s>>>(la, theta, seg_off, tile_start, A, lda, Zp, ldp, C, ldc,
                                                        C2, Ze, lde);
    } else {
        k_gemm<B_TRANS, PRO, EPI, 128><<<g, 256, 0, s>>>(la, theta, seg_off, tile_start, A, lda, Zp, ldp, C, ldc,
                                                         C2, Ze, lde);
    }
}

cudaError_t mlp_tiles(const MlpPlan& p, const int32_t* seg_off, int32_t* tile_start, cudaStream_t s, int* launches)
{
    k_tiles<<<1, 32, 0, s>>>(p.S, seg_off, tile_start);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t mlp_forward(const MlpPlan& p, const MlpBuffers& b, const float* theta, int64_t N, cudaStream_t s,
                        int* launches, int l0)
{
    for (int l = l0; l < p.L; ++l) {
        LayerArgs la = layer_args(p, l, false);
        const float* Ain = l == 0 ? b.G : b.A[l];
        const int lda = p.ld[l];
        launch_gemm<true, PRO_NONE, EPI_FWD>(p, N, p.ld[l + 1], s, la, theta, b.seg_off, b.tile_start, Ain, lda,
                                             nullptr, 0, b.Z[l + 1], p.ld[l + 1], b.A[l + 1], nullptr, 0);
        ++*launches;
    }
    return cudaGetLastError();
}

cudaError_t mlp_input_grad(const MlpPlan& p, const MlpBuffers& b, const float* theta, int64_t N, float* g,
                           cudaStream_t s, int* launches, float** ab1, bool seeded)
{
    // seed dE/da_L = 1 (unless given), then a_{l-1}bar = (a_l bar * act'(z_l)) W_l
    if (!seeded) {
        k_seed<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, p.ld[p.L], nullptr, 0.f, b.Ab, nullptr);
        ++*launches;
    }
    float* cur = b.Ab;
    float* nxt = b.Ab2;
    const int lstop = ab1 ? 1 : 0;
    for (int l = p.L - 1; l >= lstop; --l) {
        LayerArgs la = layer_args(p, l, true);
        float* out = l == 0 ? g : nxt;
        const int ldo = p.ld[l];
        launch_gemm<false, PRO_DACT, EPI_STORE>(p, N, p.ld[l], s, la, theta, b.seg_off, b.tile_start, cur,
                                                p.ld[l + 1], b.Z[l + 1], p.ld[l + 1], out, ldo, nullptr, nullptr, 0);
        ++*launches;
        float* t = cur; cur = out; nxt = t;
    }
    if (ab1) *ab1 = cur;
    return cudaGetLastError();
}

cudaError_t mlp_param_grad(const MlpPlan& p, const MlpBuffers& b, const float* theta, int64_t N,
                           const float* wdot, const float* alpha_rows, float* dtheta, cudaStream_t s,
                           int* launches, bool tan_tc, const WgradTc* wtc, MlpGradPart part)
{
    // forward tangent along wdot: zdot_l = adot_{l-1} W_l^T, adot_l = act'(z_l) zdot_l
    for (int l = tan_tc ? 1 : 0; l < p.L && part != MLP_GRAD_REVERSE_SEEDED; ++l) {
        LayerArgs la = layer_args(p, l, false);
        const float* Ain = l == 0 ? wdot : b.Ad[l];
        launch_gemm<true, PRO_NONE, EPI_TAN>(p, N, p.ld[l + 1], s, la, theta, b.seg_off, b.tile_start, Ain,
                                             p.ld[l], nullptr, 0, b.Zd[l + 1], p.ld[l + 1], b.Ad[l + 1], b.Z[l + 1],
                                             p.ld[l + 1]);
        ++*launches;
    }
    if (part == MLP_GRAD_TANGENT) return cudaGetLastError();
    // reverse pass: seeds abar_L = alpha, adotbar_L = -1 (unless given)
    if (part != MLP_GRAD_REVERSE_SEEDED) {
        k_seed<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, p.ld[p.L], alpha_rows, -1.f, b.Ab, b.Adb);
        ++*launches;
    }
    for (int l = p.L - 1; l >= 0; --l) {
        const int ldl = p.ld[l + 1];
        k_layer_adjoint<<<(unsigned)((N * ldl + 255) / 256), 256, 0, s>>>(
            layer_args(p, l, false), b.seg_off, N, ldl, b.Ab, b.Adb, b.Z[l + 1], b.Zd[l + 1], b.Zb, b.Zdb);
        ++*launches;
        // weight gradient of layer l+1
        LayerArgs lw = layer_args(p, l, false);
        const float* Ain = l == 0 ? b.G : b.A[l];
        const float* Adin = l == 0 ? wdot : b.Ad[l];
        if (wtc && wtc->ws) {
            cudaError_t e = tf32_wgrad(p, b, N, wtc->ws, wtc->mask, l, Ain, Adin, dtheta, wtc->status, s, launches);
            if (e != cudaSuccess) return e;
        } else {
            int kmax = 0, nmax = 0;
            for (int q = 0; q < p.S; ++q) { kmax = max(kmax, lw.K[q]); nmax = max(nmax, lw.N[q]); }
            dim3 gw((unsigned)((nmax + kBM - 1) / kBM), (unsigned)((kmax + 1 + kBN - 1) / kBN),
                    (unsigned)(p.S * b.splits));
            k_wgrad<<<gw, 256, 0, s>>>(lw, b.seg_off, b.splits, b.Zb, Ain, ldl, p.ld[l], b.Zdb, Adin, b.part, p.P);
            ++*launches;
        }
        if (l > 0) {
            // abar_{l} = Zb W_{l+1}, adotbar_{l} = Zdb W_{l+1}
            LayerArgs la = layer_args(p, l, true);
            launch_gemm<false, PRO_NONE, EPI_STORE>(p, N, p.ld[l], s, la, theta, b.seg_off, b.tile_start, b.Zb,
                                                    ldl, nullptr, 0, b.Ab, p.ld[l], nullptr, nullptr, 0);
            launch_gemm<false, PRO_NONE, EPI_STORE>(p, N, p.ld[l], s, la, theta, b.seg_off, b.tile_start, b.Zdb,
                                                    ldl, nullptr, 0, b.Adb, p.ld[l], nullptr, nullptr, 0);
            *launches += 2;
        }
    }
    if (!(wtc && wtc->ws)) {
        k_reduce_splits<<<(unsigned)((p.P + 255) / 256), 256, 0, s>>>(p.P, b.splits, b.part, dtheta);
        ++*launches;
    }
    return cudaGetLastError();
}

// E_rows[r] = A_L[r][0]
__global__ void k_take_energy(int64_t N, int ld, const float* __restrict__ AL, float* __restrict__ E_rows)
{
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < N) E_rows[r] = AL[r * ld];
}

cudaError_t mlp_energy_rows(const MlpPlan& p, const MlpBuffers& b, int64_t N, float* E_rows, cudaStream_t s,
                            int* launches)
{
    k_take_energy<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, p.ld[p.L], b.A[p.L], E_rows);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace panna
