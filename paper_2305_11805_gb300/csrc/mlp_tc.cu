// Per-species networks (Eq. 1) on the 5th-generation tensor cores: BF16 operands, FP32
// accumulation in tensor memory (TMEM), operands staged by TMA.
//
// One GEMM kernel, C[rows, N] = A[rows, K] B_s[N, K]^T, serves every layer:
//   forward  Z_{l+1} = A_l W_l^T (+ b_l), A_{l+1} = act(Z_{l+1})       (B = W_l, K-major)
//   backward abar_l  = zbar_{l+1} W_l,   zbar_l = abar_l * act'(Z_l)    (B = W_l^T, K-major)
//            g       = zbar_1 W_0  (input gradient dE/dG, FP32 out)
// Rows are atoms in species order; a CTA owns one 128-row tile of one species (tile
// table on the device) and one N tile of up to 256 columns.
//
// CTA of 6 warps: warp 0 issues TMA loads into a 4-stage ring (mbarrier full/empty),
// warp 1 owns the TMEM allocation and one lane issues tcgen05.mma (M = 128, N = BN,
// K = 16 per instruction, 4 per 64-wide K chunk) and tcgen05.commit; warps 2..5 read the
// accumulator with tcgen05.ld (each warp its 32-lane quarter) and run the epilogue.
// Every wait is bounded: on time-out the CTA sets PANNA_ERR_TIMEOUT, drains what it
// issued, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <stdint.h>
#include <string.h>

#include "mlp.cuh"

namespace panna {

namespace {

constexpr int kTcBM = 128, kTcBK = 64;
constexpr int kTcThreads = 192;
constexpr uint32_t kTmemCols = 256;
constexpr long long kSpinLimit = 1ll << 25;
constexpr uint32_t kTileA = kTcBM * kTcBK * 2;           // 16 KiB: one 128 x 64 BF16 tile

// Pipeline geometry.  Plain: one BF16 copy of each operand, N tile up to 256, 4 stages.
// Split (hi + lo BF16 pairs, three MMAs per K step): N tile up to 128, 3 stages.
template <bool SPLIT>
struct TcCfg {
    static constexpr int kMaxBN = SPLIT ? 128 : 256;
    static constexpr int kStages = SPLIT ? 3 : 4;
    static constexpr int kParts = SPLIT ? 2 : 1;
    static constexpr uint32_t kStageA = kParts * kTileA;
    static constexpr uint32_t kTileB = kMaxBN * kTcBK * 2;
    static constexpr uint32_t kStageB = kParts * kTileB;
    static constexpr size_t kSmem = 1024 + kStages * (kStageA + kStageB) + 256;
};

enum { TC_FWD = 1, TC_BWD_MID = 2, TC_BWD_OUT = 3 };

struct TcArgs {
    int S;
    int N[kMaxSpecies];        // valid output columns per species
    int K;                     // reduction length (TMA zero-fills past the tensor edge)
    int BN;                    // N tile, multiple of 16, <= 256
    int n_pad;                 // rows per species in the stacked B operand
    int act[kMaxSpecies];      // FWD: activation of this layer; BWD_MID: of the layer whose Z is read
    const float* bias;         // FWD: [S * n_pad]
    float* outF; int ldF;      // FWD: Z (FP32); BWD_OUT: g (FP32)
    __nv_bfloat16* outH; int ldH;  // FWD: act(Z); BWD_MID: zbar (BF16, hi part when split)
    __nv_bfloat16* outL;           // split: lo part, same layout as outH
    const float* Zin; int ldZ;     // BWD_MID: Z for act'
    const int32_t* seg_off;
    const int32_t* tile_start;
    DevStatus* status;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// bounded wait on a phase; false on time-out or (when abort_flag is given) once another
// role has aborted
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag)
{
    for (long long it = 0; it < kSpinLimit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (abort_flag && (it & 255) == 255 && *abort_flag) return false;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
                 : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

// Shared-memory matrix descriptor: K-major operand tile written by TMA with 128-byte
// swizzle (rows of 64 BF16 = 128 B, 8-row atoms of 1024 B stacked along M/N).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address
    d |= (uint64_t)1 << 16;                     // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                     // descriptor version
    d |= (uint64_t)2 << 61;                     // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major, M x N.
__device__ __forceinline__ uint32_t idesc_bf16(uint32_t M, uint32_t N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

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

__device__ __forceinline__ void store_split(__nv_bfloat16* hi, __nv_bfloat16* lo, size_t idx, float v)
{
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[idx] = h;
    if (lo) lo[idx] = __float2bfloat16_rn(v - __bfloat162float(h));
}

template <int EPI, bool SPLIT>
__global__ void __launch_bounds__(kTcThreads, 1)
k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
          const __grid_constant__ CUtensorMap tmA2, const __grid_constant__ CUtensorMap tmB2, TcArgs a)
{
    using Cfg = TcCfg<SPLIT>;
    constexpr int kStages = Cfg::kStages;
    extern __shared__ unsigned char smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;                                  // [stage][part] 128 x 64 tiles
    uint8_t* sB = smem + kStages * Cfg::kStageA;         // [stage][part] BN x 64 tiles
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + kStages * Cfg::kStageB);
    uint64_t* empty = full + kStages;
    uint64_t* accf = empty + kStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accf + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile = blockIdx.x;
    if (tile >= a.tile_start[a.S]) return;              // whole CTA: no barrier touched yet
    int s = 0;
    while (tile >= a.tile_start[s + 1]) ++s;
    const int n0 = blockIdx.y * a.BN;
    if (n0 >= a.N[s]) return;
    const int row0 = a.seg_off[s] + (tile - a.tile_start[s]) * kTcBM;
    const int rend = a.seg_off[s + 1];
    const int nk = (a.K + kTcBK - 1) / kTcBK;

    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) { mbar_init(full + i, 1); mbar_init(empty + i, 1); }
        mbar_init(accf, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(tmem_slot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t bytes = Cfg::kParts * (kTileA + (uint32_t)a.BN * kTcBK * 2);

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int kc = 0; kc < nk; ++kc) {
                const int st = kc % kStages;
                const uint32_t ph = (uint32_t)(kc / kStages) & 1u;
                if (!mbar_wait(empty + st, ph ^ 1u, abort_flag)) { *abort_flag = 1; break; }
                mbar_expect_tx(full + st, bytes);
                uint8_t* a_st = sA + st * Cfg::kStageA;
                uint8_t* b_st = sB + st * Cfg::kStageB;
                tma_load_2d(a_st, &tmA, kc * kTcBK, row0, full + st);
                tma_load_2d(b_st, &tmB, kc * kTcBK, s * a.n_pad + n0, full + st);
                if (SPLIT) {
                    tma_load_2d(a_st + kTileA, &tmA2, kc * kTcBK, row0, full + st);
                    tma_load_2d(b_st + Cfg::kTileB, &tmB2, kc * kTcBK, s * a.n_pad + n0, full + st);
                }
                ++issued;
            }
            // never leave with copies in flight: wait (bounded) for the last ones to land
            for (int kc = issued > kStages ? issued - kStages : 0; kc < issued; ++kc)
                mbar_wait(full + kc % kStages, (uint32_t)(kc / kStages) & 1u, nullptr);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(kTcBM, (uint32_t)a.BN);
            bool ok = true;
            for (int kc = 0; kc < nk; ++kc) {
                const int st = kc % kStages;
                const uint32_t ph = (uint32_t)(kc / kStages) & 1u;
                if (!mbar_wait(full + st, ph, abort_flag)) { *abort_flag = 1; ok = false; break; }
                tc_fence_after();
                const uint32_t a0 = smem_u32(sA + st * Cfg::kStageA), b0 = smem_u32(sB + st * Cfg::kStageB);
#pragma unroll
                for (int kk = 0; kk < kTcBK / 16; ++kk) {
                    const uint64_t ah = sw128_desc(a0 + kk * 32), bh = sw128_desc(b0 + kk * 32);
                    tc_mma(tmem, ah, bh, idesc, (kc | kk) ? 1u : 0u);
                    if (SPLIT) {
                        // hi*lo and lo*hi terms; lo*lo is below the accumulation precision
                        tc_mma(tmem, ah, sw128_desc(b0 + Cfg::kTileB + kk * 32), idesc, 1u);
                        tc_mma(tmem, sw128_desc(a0 + kTileA + kk * 32), bh, idesc, 1u);
                    }
                }
                tc_commit(empty + st);
            }
            tc_commit(accf);   // arrives once every MMA issued above has completed
            if (!ok) mbar_wait(accf, 0, nullptr);   // no TMEM release under running MMAs
        }
    } else {
        const int q = warp & 3;                    // TMEM lane quarter of this warp
        const int r = row0 + q * 32 + lane;        // this thread's row
        if (mbar_wait(accf, 0, abort_flag)) {
            tc_fence_after();
            const int Ns = a.N[s];
            for (int c0 = 0; c0 < a.BN; c0 += 16) {
                float v[16];
                tc_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
                if (r >= rend) continue;
                const int nb = n0 + c0;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int n = nb + j;
                    if (n >= Ns) break;
                    if (EPI == TC_FWD) {
                        const float z = v[j] + a.bias[s * a.n_pad + n];
                        a.outF[(size_t)r * a.ldF + n] = z;
                        store_split(a.outH, SPLIT ? a.outL : nullptr, (size_t)r * a.ldH + n, act_f(a.act[s], z));
                    } else if (EPI == TC_BWD_MID) {
                        const float zb = v[j] * act_d1(a.act[s], a.Zin[(size_t)r * a.ldZ + n]);
                        store_split(a.outH, SPLIT ? a.outL : nullptr, (size_t)r * a.ldH + n, zb);
                    } else {
                        a.outF[(size_t)r * a.ldF + n] = v[j];
                    }
                }
            }
        } else {
            *abort_flag = 1;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) set_status(a.status, PANNA_ERR_TIMEOUT, tile);
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

// ------------------------------------------------------------------ helper kernels

__global__ void k_tiles128(int S, const int32_t* __restrict__ seg_off, int32_t* __restrict__ tile_start)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int t = 0;
        for (int s = 0; s < S; ++s) {
            tile_start[s] = t;
            t += (seg_off[s + 1] - seg_off[s] + kTcBM - 1) / kTcBM;
        }
        tile_start[S] = t;
    }
}

__global__ void k_to_bf16(int64_t n, const float* __restrict__ x, __nv_bfloat16* __restrict__ hi,
                          __nv_bfloat16* __restrict__ lo)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) store_split(hi, lo, i, x[i]);
}

// Stacked BF16 weights of layer l for all species:
//   fwd: out[(s*npad + n) * kpad + k] = W_s[n][k]      (n < n_out_s, k < n_in_s, else 0)
//   bwd: out[(s*npad + k) * kpad + n] = W_s[n][k]      (the transpose)
__global__ void k_stack_weights(LayerArgs la, const float* __restrict__ theta, int npad, int kpad, int transpose,
                                __nv_bfloat16* __restrict__ out, __nv_bfloat16* __restrict__ out_lo,
                                float* __restrict__ bias_out)
{
    const int64_t total = (int64_t)la.S * npad * kpad;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int s = (int)(idx / ((int64_t)npad * kpad));
    const int rr = (int)((idx / kpad) % npad);
    const int cc = (int)(idx % kpad);
    const int n_out = la.N[s], n_in = la.K[s];
    const int n = transpose ? cc : rr, k = transpose ? rr : cc;
    float v = 0.f;
    if (n < n_out && k < n_in) v = theta[la.w_off[s] + (int64_t)n * n_in + k];
    store_split(out, out_lo, idx, v);
    if (bias_out && !transpose && cc == 0) bias_out[(int64_t)s * npad + rr] = rr < n_out ? theta[la.b_off[s] + rr] : 0.f;
}

// Output layer (width 1) and the start of the backward pass, one warp per row:
//   z = sum_h w[h] act(Z[h]) + b, E = act_out(z), zbar[h] = act_out'(z) w[h] act'(Z[h]).
__global__ void k_out_layer(int S, const int32_t* __restrict__ seg_off, int64_t N, LayerArgs lo,
                            const float* __restrict__ theta,
                            const float* __restrict__ Z, int ldZ, float* __restrict__ E_rows,
                            __nv_bfloat16* __restrict__ zbar, __nv_bfloat16* __restrict__ zbar_lo, int ldzb,
                            LayerArgs lp)
{
    const int lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (r >= N || r >= seg_off[S]) return;     // rows past the last species (ghost atoms have none)
    int s = 0;
    while (s < S - 1 && r >= seg_off[s + 1]) ++s;
    const int H = lo.K[s];
    const float* w = theta + lo.w_off[s];
    const int ta = lp.act[s];
    float acc = 0.f;
    for (int h = lane; h < H; h += 32) acc = fmaf(w[h], act_f(ta, Z[r * ldZ + h]), acc);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    const float z = acc + theta[lo.b_off[s]];
    const int to = lo.act[s];
    if (lane == 0) E_rows[r] = act_f(to, z);
    const float dz = act_d1(to, z);
    for (int h = lane; h < ldzb; h += 32) {
        float v = 0.f;
        if (h < H) v = dz * w[h] * act_d1(ta, Z[r * ldZ + h]);
        store_split(zbar, zbar_lo, r * ldzb + h, v);
    }
}

// ------------------------------------------------------------------ host side

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

cudaError_t get_encoder()
{
    if (g_encode) return cudaSuccess;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    return cudaSuccess;
}

// 2D BF16 tensor [rows x cols] (row stride ld elements), box [box_rows x 64], 128 B swizzle
cudaError_t make_map(CUtensorMap* m, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows)
{
    if ((reinterpret_cast<uintptr_t>(base) & 15) || (ld * 2) % 16) return cudaErrorInvalidValue;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)(rows > 0 ? rows : 1)};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    cuuint32_t box[2] = {(cuuint32_t)kTcBK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

LayerArgs tc_layer_args(const MlpPlan& p, int l)
{
    LayerArgs la{};
    la.S = p.S;
    for (int s = 0; s < p.S; ++s) {
        la.K[s] = p.widths[s][l];
        la.N[s] = p.widths[s][l + 1];
        la.act[s] = p.acts[s][l];
        la.pact[s] = p.acts[s][l];
        la.w_off[s] = p.w_off[s][l];
        la.b_off[s] = p.b_off[s][l];
    }
    return la;
}

int tc_bn(int n, int max_bn) { int t = (n + max_bn - 1) / max_bn; return round_up((n + t - 1) / t, 16); }

template <int EPI, bool SPLIT>
cudaError_t launch_tc(const CUtensorMap* m, const TcArgs& ta, int64_t N, int nmax, cudaStream_t s)
{
    const int smem = (int)TcCfg<SPLIT>::kSmem;
    cudaError_t e = cudaFuncSetAttribute(k_tc_gemm<EPI, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((N + kTcBM - 1) / kTcBM + ta.S), (unsigned)((nmax + ta.BN - 1) / ta.BN));
    k_tc_gemm<EPI, SPLIT><<<grid, kTcThreads, smem, s>>>(m[0], m[1], m[2], m[3], ta);
    return cudaGetLastError();
}

template <int EPI>
cudaError_t launch_tc_any(bool split, const CUtensorMap* m, const TcArgs& ta, int64_t N, int nmax, cudaStream_t s)
{
    return split ? launch_tc<EPI, true>(m, ta, N, nmax, s) : launch_tc<EPI, false>(m, ta, N, nmax, s);
}

// Buffers of the BF16 networks, carved from one workspace block (sizing when base == nullptr).
struct TcBufs {
    int32_t* tiles128;
    __nv_bfloat16* G16[2];                       // hi, lo
    __nv_bfloat16* A16[kMaxLayers + 1][2];
    __nv_bfloat16* Zb16[kMaxLayers + 1][2];
    __nv_bfloat16* Wf[kMaxLayers][2];
    __nv_bfloat16* Wb[kMaxLayers][2];
    float* bias[kMaxLayers];
    int ldh[kMaxLayers + 1];
    int npf[kMaxLayers], npb[kMaxLayers], bnf[kMaxLayers], bnb[kMaxLayers];
};

size_t tc_carve(const MlpPlan& p, int64_t N, bool split, char* base, TcBufs& t)
{
    size_t off = 0;
    auto take = [&](size_t n) {
        void* q = base ? base + off : nullptr;
        off += (n + 255) & ~(size_t)255;
        return q;
    };
    const int parts = split ? 2 : 1;
    const int max_bn = split ? TcCfg<true>::kMaxBN : TcCfg<false>::kMaxBN;
    t.tiles128 = static_cast<int32_t*>(take((kMaxSpecies + 1) * sizeof(int32_t)));
    t.ldh[0] = round_up(p.ld[0], 8);
    for (int q = 0; q < 2; ++q) t.G16[q] = q < parts ? static_cast<__nv_bfloat16*>(take((size_t)N * t.ldh[0] * 2)) : nullptr;
    for (int l = 1; l < p.L; ++l) {
        t.ldh[l] = round_up(p.ld[l], 8);
        for (int q = 0; q < 2; ++q) {
            t.A16[l][q] = q < parts ? static_cast<__nv_bfloat16*>(take((size_t)N * t.ldh[l] * 2)) : nullptr;
            t.Zb16[l][q] = q < parts ? static_cast<__nv_bfloat16*>(take((size_t)N * t.ldh[l] * 2)) : nullptr;
        }
    }
    for (int l = 0; l < p.L - 1; ++l) {
        const int no = p.ld[l + 1], ni = p.ld[l];
        t.bnf[l] = tc_bn(no, max_bn); t.bnb[l] = tc_bn(ni, max_bn);
        t.npf[l] = round_up(no, t.bnf[l]); t.npb[l] = round_up(ni, t.bnb[l]);
        for (int q = 0; q < 2; ++q) {
            t.Wf[l][q] = q < parts ? static_cast<__nv_bfloat16*>(take((size_t)p.S * t.npf[l] * round_up(ni, 8) * 2)) : nullptr;
            t.Wb[l][q] = q < parts ? static_cast<__nv_bfloat16*>(take((size_t)p.S * t.npb[l] * round_up(no, 8) * 2)) : nullptr;
        }
        t.bias[l] = static_cast<float*>(take((size_t)p.S * t.npf[l] * 4));
    }
    return off + 4096;
}

// 2D BF16 tensor [rows x cols] (row stride ld elements), box [box_rows x 64], 128 B swizzle
cudaError_t make_maps(CUtensorMap* m, __nv_bfloat16* const* base, int parts, int64_t rows, int64_t cols, int64_t ld,
                      int box_rows)
{
    for (int q = 0; q < parts; ++q) {
        cudaError_t e = make_map(&m[q], base[q], rows, cols, ld, box_rows);
        if (e != cudaSuccess) return e;
    }
    if (parts == 1) m[1] = m[0];
    return cudaSuccess;
}

}  // namespace

size_t tc_workspace_bytes(const MlpPlan& p, int64_t N, bool split)
{
    TcBufs t;
    return tc_carve(p, N, split, nullptr, t);
}

// Energies (E_rows) and input gradients g = dE/dG (FP32 rows) of all rows with BF16 tensor-core
// GEMMs (FP32 accumulation).  split: every BF16 operand is carried as a hi + lo pair and each
// product takes three MMAs (hi*hi + hi*lo + lo*hi), about 16 significant bits per operand.
// G rows in FP32 are converted first.  Needs at least one hidden layer.
cudaError_t mlp_bf16_energy_grad(const MlpPlan& p, const MlpBuffers& b, const float* theta, int64_t N, void* ws,
                                 bool split, float* E_rows, float* g, DevStatus* status, cudaStream_t s,
                                 int* launches)
{
    if (p.L < 2) return cudaErrorNotSupported;
    cudaError_t e = get_encoder();
    if (e != cudaSuccess) return e;
    TcBufs t;
    tc_carve(p, N, split, static_cast<char*>(ws), t);
    const int parts = split ? 2 : 1;
    if (t.ldh[0] != p.ld[0]) return cudaErrorNotSupported;   // descriptor width not a multiple of 8
    k_tiles128<<<1, 32, 0, s>>>(p.S, b.seg_off, t.tiles128);
    ++*launches;
    for (int l = 0; l < p.L - 1; ++l) {
        const int no = p.ld[l + 1], ni = p.ld[l];
        LayerArgs la = tc_layer_args(p, l);
        int64_t tf = (int64_t)p.S * t.npf[l] * round_up(ni, 8);
        k_stack_weights<<<(unsigned)((tf + 255) / 256), 256, 0, s>>>(la, theta, t.npf[l], round_up(ni, 8), 0,
                                                                    t.Wf[l][0], t.Wf[l][1], t.bias[l]);
        int64_t tb = (int64_t)p.S * t.npb[l] * round_up(no, 8);
        k_stack_weights<<<(unsigned)((tb + 255) / 256), 256, 0, s>>>(la, theta, t.npb[l], round_up(no, 8), 1,
                                                                    t.Wb[l][0], t.Wb[l][1], nullptr);
        *launches += 2;
    }
    // padding columns of the BF16 operands meet zero weights, but must not hold NaN
    for (int l = 1; l < p.L; ++l)
        for (int q = 0; q < parts; ++q) {
            e = cudaMemsetAsync(t.A16[l][q], 0, (size_t)N * t.ldh[l] * 2, s);
            if (e == cudaSuccess) e = cudaMemsetAsync(t.Zb16[l][q], 0, (size_t)N * t.ldh[l] * 2, s);
            if (e != cudaSuccess) return e;
        }
    k_to_bf16<<<(unsigned)((N * t.ldh[0] + 255) / 256), 256, 0, s>>>(N * t.ldh[0], b.G, t.G16[0], t.G16[1]);
    ++*launches;

    TcArgs base{};
    base.S = p.S;
    base.seg_off = b.seg_off;
    base.tile_start = t.tiles128;
    base.status = status;
    CUtensorMap maps[4];   // A hi, B hi, A lo, B lo
    // forward through the hidden layers
    for (int l = 0; l < p.L - 1; ++l) {
        CUtensorMap mA[2], mB[2];
        __nv_bfloat16* const* Ain = l == 0 ? t.G16 : t.A16[l];
        e = make_maps(mA, Ain, parts, N, p.ld[l], t.ldh[l], kTcBM);
        if (e == cudaSuccess)
            e = make_maps(mB, t.Wf[l], parts, (int64_t)p.S * t.npf[l], p.ld[l], round_up(p.ld[l], 8), t.bnf[l]);
        if (e != cudaSuccess) return e;
        maps[0] = mA[0]; maps[1] = mB[0]; maps[2] = mA[1]; maps[3] = mB[1];
        TcArgs ta = base;
        for (int q = 0; q < p.S; ++q) { ta.N[q] = p.widths[q][l + 1]; ta.act[q] = p.acts[q][l]; }
        ta.K = p.ld[l];
        ta.BN = t.bnf[l];
        ta.n_pad = t.npf[l];
        ta.bias = t.bias[l];
        ta.outF = b.Z[l + 1]; ta.ldF = p.ld[l + 1];
        ta.outH = t.A16[l + 1][0]; ta.outL = t.A16[l + 1][1]; ta.ldH = t.ldh[l + 1];
        e = launch_tc_any<TC_FWD>(split, maps, ta, N, p.ld[l + 1], s);
        if (e != cudaSuccess) return e;
        ++*launches;
    }
    // output layer and the first backward step
    {
        LayerArgs lo = tc_layer_args(p, p.L - 1);
        LayerArgs lp = tc_layer_args(p, p.L - 2);
        k_out_layer<<<(unsigned)((N + 7) / 8), 256, 0, s>>>(p.S, b.seg_off, N, lo, theta, b.Z[p.L - 1],
                                                           p.ld[p.L - 1], E_rows, t.Zb16[p.L - 1][0],
                                                           t.Zb16[p.L - 1][1], t.ldh[p.L - 1], lp);
        ++*launches;
    }
    // backward through the hidden layers down to the input gradient
    for (int l = p.L - 2; l >= 0; --l) {
        CUtensorMap mA[2], mB[2];
        e = make_maps(mA, t.Zb16[l + 1], parts, N, p.ld[l + 1], t.ldh[l + 1], kTcBM);
        if (e == cudaSuccess)
            e = make_maps(mB, t.Wb[l], parts, (int64_t)p.S * t.npb[l], p.ld[l + 1], round_up(p.ld[l + 1], 8),
                          t.bnb[l]);
        if (e != cudaSuccess) return e;
        maps[0] = mA[0]; maps[1] = mB[0]; maps[2] = mA[1]; maps[3] = mB[1];
        TcArgs ta = base;
        for (int q = 0; q < p.S; ++q) ta.N[q] = p.widths[q][l];
        ta.K = p.ld[l + 1];
        ta.BN = t.bnb[l];
        ta.n_pad = t.npb[l];
        if (l > 0) {
            for (int q = 0; q < p.S; ++q) ta.act[q] = p.acts[q][l - 1];
            ta.Zin = b.Z[l]; ta.ldZ = p.ld[l];
            ta.outH = t.Zb16[l][0]; ta.outL = t.Zb16[l][1]; ta.ldH = t.ldh[l];
            e = launch_tc_any<TC_BWD_MID>(split, maps, ta, N, p.ld[l], s);
        } else {
            ta.outF = g; ta.ldF = p.ld[0];
            e = launch_tc_any<TC_BWD_OUT>(split, maps, ta, N, p.ld[0], s);
        }
        if (e != cudaSuccess) return e;
        ++*launches;
    }
    return cudaGetLastError();
}

}  // namespace panna
