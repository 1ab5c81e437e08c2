// Per-species networks (Eq. 1) on the 5th-generation tensor cores: BF16 or TF32 operands,
// FP32 accumulation in tensor memory (TMEM), operands staged by TMA.  Either operand type
// may be carried as a hi + lo pair (three MMAs per product, hi*hi + hi*lo + lo*hi): BF16
// pairs keep about 16 significant bits, TF32 pairs about 22 (FP32-class results).
//
// One GEMM kernel, C[rows, N] = A[rows, K] B_s[N, K]^T, serves every layer:
//   forward  Z_{l+1} = A_l W_l^T (+ b_l), A_{l+1} = act(Z_{l+1})       (B = W_l, K-major)
//   backward abar_l  = zbar_{l+1} W_l,   zbar_l = abar_l * act'(Z_l)    (B = W_l^T, K-major)
//            g       = zbar_1 W_0  (input gradient dE/dG, FP32 out)
//   tangent  zdot_1  = Gdot W_0^T, adot_1 = act'(Z_1) zdot_1             (FP32 out)
//   weights  dW_0    = zbar_1^T G + zdotbar_1^T Gdot  (sum over atoms: operands transposed
//            so that atoms run along K, each species padded to 32 atoms; one CTA per
//            (species, chunk of atoms, 128 outputs, N tile), partial sums reduced in order)
// Rows are atoms in species order; a CTA owns one 128-row tile of one species (tile
// table on the device) and one N tile of up to 256 columns.
//
// CTA of 10 warps: warp 0 issues TMA loads into a 2-4 stage ring (mbarrier full/empty),
// warp 1 owns the TMEM allocation and one lane issues tcgen05.mma (M = 128, N = BN,
// K = 16 BF16 or 8 TF32 per instruction, 4 per 128-byte K chunk) and tcgen05.commit; warps 2..9
// read the accumulator with tcgen05.ld (two warps per 32-lane quarter) and run the epilogue.
// Every wait is bounded: on time-out the CTA sets PANNA_ERR_TIMEOUT, drains what it
// issued, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <stdint.h>
#include <algorithm>
#include <string.h>

#include "mlp.cuh"

namespace panna {

namespace {

constexpr int kTcBM = 128, kTcBK = 64;   // kTcBK: BF16 elements per 128-byte K chunk (32 for TF32)
constexpr int kTcEpiWarps = 8;                          // two per TMEM lane quarter
constexpr int kTcThreads = 64 + 32 * kTcEpiWarps;
constexpr uint32_t kTmemCols = 256;
constexpr long long kSpinLimit = 1ll << 25;
constexpr uint32_t kTileA = kTcBM * kTcBK * 2;           // 16 KiB: one 128 x 64 BF16 tile

// Pipeline geometry by the number of parts each operand is carried in:
//   1: plain, N tile up to 256, 4 stages;
//   2: hi + lo (three MMAs per K step), N tile up to 128, 3 stages;
//   3: hi + mid + lo, an exact split of FP32 into TF32 (six MMAs per K step: every cross term
//      above 2^-32 of the product), N tile up to 128, 2 stages.
template <int PARTS>
struct TcCfg {
    static constexpr int kMaxBN = PARTS == 1 ? 256 : 128;
    static constexpr int kStages = PARTS == 1 ? 4 : (PARTS == 2 ? 3 : 2);
    static constexpr int kParts = PARTS;
    static constexpr uint32_t kStageA = kParts * kTileA;
    static constexpr uint32_t kTileB = kMaxBN * kTcBK * 2;
    static constexpr uint32_t kStageB = kParts * kTileB;
    static constexpr size_t kSmem = 1024 + kStages * (kStageA + kStageB) + 256;
    // the persistent kernel adds a 2 KB staging tile per epilogue warp for its FP32 outputs
    static constexpr size_t kSmemP = kSmem + 2048 * 8;
};

enum { TC_FWD = 1, TC_BWD_MID = 2, TC_BWD_OUT = 3, TC_FWD32 = 4, TC_TAN32 = 5, TC_WGRAD = 6 };

// TMA descriptors of the parts of both operands (one kernel parameter in param space)
struct TcMaps {
    CUtensorMap a[3];
    CUtensorMap b[3];
};

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
    const float* Zin; int ldZ;     // BWD_MID, TAN32: Z for act'
    float* outA; int ldA;          // FWD32: act(Z); TAN32: act'(Z) zdot (FP32)
    // WGRAD: species-padded transposed operands, items = (species, chunk of atoms)
    const int32_t* item_start;     // [S+1]
    const int32_t* pstart;         // [S+1] padded column of each species' first atom
    int Kp;                        // column offset of the second product's operands
    int chunk;                     // atoms per item (multiple of 32)
    float* part; int ldn;          // part[(item * Mvalid + m) * ldn + n]
    int Mvalid, Nvalid;            // outputs m < Mvalid, n < Nvalid
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

template <bool TF>
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    if (TF)
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                     ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
                     : "memory");
    else
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

// Instruction descriptor: D FP32, A and B both K-major, M x N; operand format BF16
// (kind::f16, code 1) or TF32 (kind::tf32, code 2).
__device__ __forceinline__ uint32_t idesc_mma(bool tf32, uint32_t M, uint32_t N)
{
    const uint32_t fmt = tf32 ? 2u : 1u;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

// x rounded to TF32 (10 explicit mantissa bits, low 13 bits of the FP32 pattern zero)
__device__ __forceinline__ float to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// v as up to three TF32 parts: hi = tf32(v), mid = tf32(v - hi), lo = v - hi - mid.  Each
// difference is exact in FP32, and the three parts add up to v exactly (11 + 11 + at most
// 3 significant bits).  Parts whose pointer is null are not written.
__device__ __forceinline__ void store_split_tf32(float* hi, float* mid, float* lo, size_t idx, float v)
{
    const float h = to_tf32(v);
    hi[idx] = h;
    if (mid) {
        const float r = v - h;
        const float m = to_tf32(r);
        mid[idx] = m;
        if (lo) lo[idx] = to_tf32(r - m);
    }
}

struct Parts3 { float* p[3]; };   // destinations of up to three TF32 parts (null = not written)

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

template <int EPI, int PARTS, bool TF>
__global__ void __launch_bounds__(kTcThreads, 1)
k_tc_gemm(const __grid_constant__ TcMaps tm, TcArgs a)
{
    using Cfg = TcCfg<PARTS>;
    constexpr int kStages = Cfg::kStages;
    constexpr int BKE = TF ? kTcBK / 2 : kTcBK;          // elements per 128-byte K chunk
    constexpr int MMAK = TF ? 8 : 16;                    // K per instruction (32 bytes)
    extern __shared__ unsigned char smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;                                  // [stage][part] 128 x 128 B tiles
    uint8_t* sB = smem + kStages * Cfg::kStageA;         // [stage][part] BN x 128 B tiles
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + kStages * Cfg::kStageB);
    uint64_t* empty = full + kStages;
    uint64_t* accf = empty + kStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accf + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // work decode (whole-CTA returns happen before any barrier or TMEM use)
    int s = 0, row0 = 0, rend = 0, n0 = 0, m0 = 0, kbeg = 0, nkh = 0, nk = 0;
    const int item = blockIdx.x;
    if (EPI == TC_WGRAD) {
        if (item >= a.item_start[a.S]) return;
        while (item >= a.item_start[s + 1]) ++s;
        kbeg = a.pstart[s] + (item - a.item_start[s]) * a.chunk;
        const int kend = min(kbeg + a.chunk, a.pstart[s + 1]);
        nkh = (kend - kbeg) / BKE;
        nk = 2 * nkh;                                     // first product, then the second
        n0 = blockIdx.y * a.BN;
        m0 = blockIdx.z * kTcBM;
        if (nk == 0 || n0 >= a.Nvalid || m0 >= a.Mvalid) return;
    } else {
        const int tile = blockIdx.x;
        if (tile >= a.tile_start[a.S]) return;
        while (tile >= a.tile_start[s + 1]) ++s;
        n0 = blockIdx.y * a.BN;
        if (n0 >= a.N[s]) return;
        row0 = a.seg_off[s] + (tile - a.tile_start[s]) * kTcBM;
        rend = a.seg_off[s + 1];
        nk = (a.K + BKE - 1) / BKE;
    }

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
    const uint32_t bytes = Cfg::kParts * (kTileA + (uint32_t)a.BN * 128u);

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
                int ka, ra, kb, rb;
                if (EPI == TC_WGRAD) {
                    ka = kb = kc < nkh ? kbeg + kc * BKE : a.Kp + kbeg + (kc - nkh) * BKE;
                    ra = m0;
                    rb = n0;
                } else {
                    ka = kb = kc * BKE;
                    ra = row0;
                    rb = s * a.n_pad + n0;
                }
#pragma unroll
                for (int q = 0; q < PARTS; ++q) {
                    tma_load_2d(a_st + q * kTileA, &tm.a[q], ka, ra, full + st);
                    tma_load_2d(b_st + q * Cfg::kTileB, &tm.b[q], kb, rb, full + st);
                }
                ++issued;
            }
            // never leave with copies in flight: wait (bounded) for the last ones to land
            for (int kc = issued > kStages ? issued - kStages : 0; kc < issued; ++kc)
                mbar_wait(full + kc % kStages, (uint32_t)(kc / kStages) & 1u, nullptr);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_mma(TF, kTcBM, (uint32_t)a.BN);
            bool ok = true;
            for (int kc = 0; kc < nk; ++kc) {
                const int st = kc % kStages;
                const uint32_t ph = (uint32_t)(kc / kStages) & 1u;
                if (!mbar_wait(full + st, ph, abort_flag)) { *abort_flag = 1; ok = false; break; }
                tc_fence_after();
                const uint32_t a0 = smem_u32(sA + st * Cfg::kStageA), b0 = smem_u32(sB + st * Cfg::kStageB);
#pragma unroll
                for (int kk = 0; kk < BKE / MMAK; ++kk) {
                    const uint64_t a1 = sw128_desc(a0 + kk * 32), b1 = sw128_desc(b0 + kk * 32);
                    tc_mma<TF>(tmem, a1, b1, idesc, (kc | kk) ? 1u : 0u);
                    if (PARTS >= 2) {
                        // cross terms down to 2^-22 (two parts) or 2^-33 (three parts) of the product
                        const uint64_t a2 = sw128_desc(a0 + kTileA + kk * 32);
                        const uint64_t b2 = sw128_desc(b0 + Cfg::kTileB + kk * 32);
                        tc_mma<TF>(tmem, a1, b2, idesc, 1u);
                        tc_mma<TF>(tmem, a2, b1, idesc, 1u);
                        if (PARTS >= 3) {
                            const uint64_t a3 = sw128_desc(a0 + 2 * kTileA + kk * 32);
                            const uint64_t b3 = sw128_desc(b0 + 2 * Cfg::kTileB + kk * 32);
                            tc_mma<TF>(tmem, a1, b3, idesc, 1u);
                            tc_mma<TF>(tmem, a2, b2, idesc, 1u);
                            tc_mma<TF>(tmem, a3, b1, idesc, 1u);
                        }
                    }
                }
                tc_commit(empty + st);
            }
            tc_commit(accf);   // arrives once every MMA issued above has completed
            if (!ok) mbar_wait(accf, 0, nullptr);   // no TMEM release under running MMAs
        }
    } else {
        // Epilogue in two passes through shared memory (the pipeline buffers are free once
        // every MMA has completed).  Pass 1: the two warps of each TMEM lane quarter copy their
        // 32 rows into a [128][BN + 4] FP32 tile (16-byte aligned rows), alternating 16-column
        // chunks.  Pass 2: warp w sweeps rows w, w + 8, ...; each lane takes 4 consecutive
        // columns, so loads and stores of a row are contiguous (float4 where aligned).  Every
        // epilogue warp reaches the named barrier, also after a failed wait.
        const int ew = warp - 2;                   // epilogue warp 0..7
        const int q = warp & 3;                    // TMEM lane quarter (hardware: warp id mod 4)
        const int half = ew >> 2;
        const int ldt = a.BN + 4;
        float* tile_s = reinterpret_cast<float*>(smem);
        const bool ok = mbar_wait(accf, 0, abort_flag);
        if (ok) {
            tc_fence_after();
            for (int c0 = half * 16; c0 < a.BN; c0 += 32) {
                float v[16];
                tc_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
                float4* dst = reinterpret_cast<float4*>(tile_s + (q * 32 + lane) * ldt + c0);
#pragma unroll
                for (int j2 = 0; j2 < 4; ++j2) dst[j2] = make_float4(v[4 * j2], v[4 * j2 + 1], v[4 * j2 + 2], v[4 * j2 + 3]);
            }
        } else {
            *abort_flag = 1;
        }
        asm volatile("bar.sync 1, %0;" ::"r"(32 * kTcEpiWarps) : "memory");
        if (!*abort_flag) {
            const int Ns = EPI == TC_WGRAD ? a.Nvalid : a.N[s];
            for (int row = ew; row < kTcBM; row += kTcEpiWarps) {
                const int r = row0 + row, m = m0 + row;
                if (EPI == TC_WGRAD ? m >= a.Mvalid : r >= rend) continue;
                for (int col = lane * 4; col < a.BN; col += 128) {
                    const int n = n0 + col;
                    if (n >= Ns) break;
                    const float4 t4 = *reinterpret_cast<const float4*>(tile_s + row * ldt + col);
                    const float v[4] = {t4.x, t4.y, t4.z, t4.w};
                    const int nv = min(4, Ns - n);
                    if (EPI == TC_WGRAD) {
                        float* o = a.part + ((size_t)item * a.Mvalid + m) * a.ldn + n;
                        for (int j2 = 0; j2 < nv; ++j2) o[j2] = v[j2];
                        continue;
                    }
                    float o1[4], o2[4];
#pragma unroll
                    for (int j2 = 0; j2 < 4; ++j2) {
                        o1[j2] = v[j2];
                        o2[j2] = 0.f;
                        if (j2 >= nv) continue;
                        if (EPI == TC_FWD || EPI == TC_FWD32) {
                            o1[j2] = v[j2] + a.bias[s * a.n_pad + n + j2];
                            o2[j2] = act_f(a.act[s], o1[j2]);
                        } else if (EPI == TC_BWD_MID) {
                            o2[j2] = v[j2] * act_d1(a.act[s], a.Zin[(size_t)r * a.ldZ + n + j2]);
                        } else if (EPI == TC_TAN32) {
                            o2[j2] = act_d1(a.act[s], a.Zin[(size_t)r * a.ldZ + n + j2]) * v[j2];
                        }
                    }
                    if (EPI == TC_FWD || EPI == TC_FWD32 || EPI == TC_TAN32 || EPI == TC_BWD_OUT) {
                        float* o = a.outF + (size_t)r * a.ldF + n;
                        if (nv == 4 && ((reinterpret_cast<uintptr_t>(o) & 15) == 0))
                            *reinterpret_cast<float4*>(o) = make_float4(o1[0], o1[1], o1[2], o1[3]);
                        else
                            for (int j2 = 0; j2 < nv; ++j2) o[j2] = o1[j2];
                    }
                    if (EPI == TC_FWD32 || EPI == TC_TAN32) {
                        float* o = a.outA + (size_t)r * a.ldA + n;
                        if (nv == 4 && ((reinterpret_cast<uintptr_t>(o) & 15) == 0))
                            *reinterpret_cast<float4*>(o) = make_float4(o2[0], o2[1], o2[2], o2[3]);
                        else
                            for (int j2 = 0; j2 < nv; ++j2) o[j2] = o2[j2];
                    }
                    if (EPI == TC_FWD || EPI == TC_BWD_MID) {
                        for (int j2 = 0; j2 < nv; ++j2)
                            store_split(a.outH, PARTS >= 2 ? a.outL : nullptr, (size_t)r * a.ldH + n + j2, o2[j2]);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) set_status(a.status, PANNA_ERR_TIMEOUT, blockIdx.x);
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

__device__ __forceinline__ void store_parts(__nv_bfloat16* hi, __nv_bfloat16* lo, __nv_bfloat16*, size_t idx, float v)
{
    store_split(hi, lo, idx, v);
}
__device__ __forceinline__ void store_parts(float* hi, float* mid, float* lo, size_t idx, float v)
{
    store_split_tf32(hi, mid, lo, idx, v);
}

// rows x cols FP32 (row stride lds) -> TF32 parts (row stride ldo, zero padding columns)
__global__ void k_split_tf32(int64_t rows, int cols, int lds, int ldo, const float* __restrict__ x, Parts3 o)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * ldo) return;
    const int64_t r = i / ldo;
    const int c = (int)(i % ldo);
    store_split_tf32(o.p[0], o.p[1], o.p[2], (size_t)i, c < cols ? x[(size_t)r * lds + c] : 0.f);
}

// Padded atom columns for the weight gradient: species s owns columns
// pstart[s] .. pstart[s] + round_up(n_s, 32) - 1, cut into items of `chunk` columns.
__global__ void k_tf32_items(int S, const int32_t* __restrict__ seg_off, int chunk, int32_t* __restrict__ pstart,
                             int32_t* __restrict__ item_start)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int p = 0, it = 0;
        for (int s = 0; s < S; ++s) {
            pstart[s] = p;
            item_start[s] = it;
            const int len = (seg_off[s + 1] - seg_off[s] + 31) / 32 * 32;
            p += len;
            it += (len + chunk - 1) / chunk;
        }
        pstart[S] = p;
        item_start[S] = it;
    }
}

struct Widths { int n[kMaxSpecies]; };

// Transposed TF32 pairs with atoms along columns:
//   dst[f * ldT + col_off + pstart[s] + (r - seg_off[s])] = src[r * lds + f]  for f < width_s,
// 1 in row f == ones_row (the bias input) for every atom, 0 elsewhere (padding atoms, f past
// the species' width, rows up to frows).  One CTA moves a 32 x 32 tile through shared memory.
__global__ void __launch_bounds__(256)
k_transpose_split(const float* __restrict__ src, int lds, int S, const int32_t* __restrict__ seg_off,
                  const int32_t* __restrict__ pstart, Widths w, int frows, int ones_row, Parts3 o, int64_t ldT,
                  int64_t col_off)
{
    __shared__ float tile[32][33];
    const int p0 = blockIdx.x * 32;
    if (p0 >= pstart[S]) return;
    int s = 0;
    while (p0 >= pstart[s + 1]) ++s;
    const int f0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int cnt = seg_off[s + 1] - seg_off[s];
    for (int pp = ty; pp < 32; pp += 8) {
        const int loc = p0 - pstart[s] + pp;
        const int f = f0 + tx;
        float v = 0.f;
        if (loc < cnt) {
            if (f < w.n[s]) v = src[(size_t)(seg_off[s] + loc) * lds + f];
            else if (f == ones_row) v = 1.f;
        }
        tile[pp][tx] = v;
    }
    __syncthreads();
    for (int ff = ty; ff < 32; ff += 8) {
        const int f = f0 + ff;
        if (f >= frows) break;
        store_split_tf32(o.p[0], o.p[1], o.p[2], (size_t)f * ldT + col_off + p0 + tx, tile[tx][ff]);
    }
}

// Weight gradient of a narrow layer (M x (K+1) <= 8192 outputs) straight from the row-major
// adjoints Zb, Zdb [rows, M] and inputs A, Ad [rows, K]: one CTA per (item = species chunk of
// atoms, split of that chunk); every thread owns up to 32 outputs o = m (K+1) + n (n == K: the
// bias), rows pass through shared memory 32 at a time.  The partial of (item, split) goes to
// part[(item * splits + split) * M (K+1) + o], so item order stays the reduction order.
constexpr int kSmallRows = 32, kSmallOut = 32;
__global__ void __launch_bounds__(256)
k_wgrad_small(int S, const int32_t* __restrict__ seg_off, const int32_t* __restrict__ item_start, int chunk,
              int splits, int M, int K, const float* __restrict__ Zb, const float* __restrict__ Zdb,
              const float* __restrict__ A, const float* __restrict__ Ad, float* __restrict__ part)
{
    extern __shared__ float sh[];
    const int item = blockIdx.x;
    if (item >= item_start[S]) return;
    int s = 0;
    while (item >= item_start[s + 1]) ++s;
    const int per = (chunk / splits + kSmallRows - 1) / kSmallRows * kSmallRows;
    const int c0 = (item - item_start[s]) * chunk + blockIdx.y * per;
    const int cend = min((item - item_start[s] + 1) * chunk, c0 + per);
    const int cnt = seg_off[s + 1] - seg_off[s];
    const int a0 = seg_off[s] + min(cnt, c0), a1 = seg_off[s] + min(cnt, cend);
    float* sZ = sh;
    float* sZd = sZ + kSmallRows * M;
    float* sA = sZd + kSmallRows * M;
    float* sAd = sA + kSmallRows * K;
    const int O = M * (K + 1);
    const int tid = threadIdx.x;
    float acc[kSmallOut];
#pragma unroll
    for (int j = 0; j < kSmallOut; ++j) acc[j] = 0.f;
    for (int r0 = a0; r0 < a1; r0 += kSmallRows) {
        const int nr = min(kSmallRows, a1 - r0);
        __syncthreads();
        for (int idx = tid; idx < kSmallRows * M; idx += 256) {
            const int rr = idx / M;
            sZ[idx] = rr < nr ? Zb[(size_t)r0 * M + idx] : 0.f;
            sZd[idx] = rr < nr ? Zdb[(size_t)r0 * M + idx] : 0.f;
        }
        for (int idx = tid; idx < kSmallRows * K; idx += 256) {
            const int rr = idx / K;
            sA[idx] = rr < nr ? A[(size_t)r0 * K + idx] : 0.f;
            sAd[idx] = rr < nr ? Ad[(size_t)r0 * K + idx] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kSmallOut; ++j) {
            const int o = j * 256 + tid;
            if (o >= O) break;
            const int m = o / (K + 1), n = o % (K + 1);
            float a = acc[j];
            if (n < K) {
                for (int rr = 0; rr < kSmallRows; ++rr)
                    a = fmaf(sZ[rr * M + m], sA[rr * K + n], fmaf(sZd[rr * M + m], sAd[rr * K + n], a));
            } else {
                for (int rr = 0; rr < kSmallRows; ++rr) a += sZ[rr * M + m];
            }
            acc[j] = a;
        }
    }
    float* out = part + ((size_t)item * splits + blockIdx.y) * O;
#pragma unroll
    for (int j = 0; j < kSmallOut; ++j) {
        const int o = j * 256 + tid;
        if (o >= O) break;
        out[o] = acc[j];
    }
}

// The same partial sums with 4 x 4 register blocks (M and K multiples of 4, (M/4)(K/4) <= 256
// blocks): thread b owns weights m in [4 (b / (K/4)), +4), n in [4 (b % (K/4)), +4), and the
// threads of the first n block also the 4 biases; per staged row it reads 4 + 4 float4 from
// shared memory for 32 FMAs (the scalar kernel above reads 4 floats per 2 FMAs).
__global__ void __launch_bounds__(256)
k_wgrad_small4(int S, const int32_t* __restrict__ seg_off, const int32_t* __restrict__ item_start, int chunk,
               int splits, int M, int K, const float* __restrict__ Zb, const float* __restrict__ Zdb,
               const float* __restrict__ A, const float* __restrict__ Ad, float* __restrict__ part)
{
    extern __shared__ __align__(16) float sh4[];
    const int item = blockIdx.x;
    if (item >= item_start[S]) return;
    int s = 0;
    while (item >= item_start[s + 1]) ++s;
    const int per = (chunk / splits + kSmallRows - 1) / kSmallRows * kSmallRows;
    const int c0 = (item - item_start[s]) * chunk + blockIdx.y * per;
    const int cend = min((item - item_start[s] + 1) * chunk, c0 + per);
    const int cnt = seg_off[s + 1] - seg_off[s];
    const int a0 = seg_off[s] + min(cnt, c0), a1 = seg_off[s] + min(cnt, cend);
    float* sZ = sh4;
    float* sZd = sZ + kSmallRows * M;
    float* sA = sZd + kSmallRows * M;
    float* sAd = sA + kSmallRows * K;
    const int tid = threadIdx.x;
    const int K4 = K >> 2, nblk = (M >> 2) * K4;
    const bool own = tid < nblk;
    const int m0 = own ? (tid / K4) * 4 : 0, n0 = own ? (tid % K4) * 4 : 0;
    float acc[4][4], bias[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        bias[a] = 0.f;
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    }
    for (int r0 = a0; r0 < a1; r0 += kSmallRows) {
        const int nr = min(kSmallRows, a1 - r0);
        __syncthreads();
        for (int idx = tid; idx < kSmallRows * M; idx += 256) {
            const int rr = idx / M;
            sZ[idx] = rr < nr ? Zb[(size_t)r0 * M + idx] : 0.f;
            sZd[idx] = rr < nr ? Zdb[(size_t)r0 * M + idx] : 0.f;
        }
        for (int idx = tid; idx < kSmallRows * K; idx += 256) {
            const int rr = idx / K;
            sA[idx] = rr < nr ? A[(size_t)r0 * K + idx] : 0.f;
            sAd[idx] = rr < nr ? Ad[(size_t)r0 * K + idx] : 0.f;
        }
        __syncthreads();
        if (own) {
            for (int rr = 0; rr < kSmallRows; ++rr) {
                const float4 z = *reinterpret_cast<const float4*>(sZ + rr * M + m0);
                const float4 zd = *reinterpret_cast<const float4*>(sZd + rr * M + m0);
                const float4 a = *reinterpret_cast<const float4*>(sA + rr * K + n0);
                const float4 ad = *reinterpret_cast<const float4*>(sAd + rr * K + n0);
                const float zv[4] = {z.x, z.y, z.z, z.w}, zdv[4] = {zd.x, zd.y, zd.z, zd.w};
                const float av[4] = {a.x, a.y, a.z, a.w}, adv[4] = {ad.x, ad.y, ad.z, ad.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    bias[i] += zv[i];
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(zv[i], av[j], fmaf(zdv[i], adv[j], acc[i][j]));
                }
            }
        }
    }
    if (!own) return;
    float* out = part + ((size_t)item * splits + blockIdx.y) * ((size_t)M * (K + 1));
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j) out[(size_t)(m0 + i) * (K + 1) + n0 + j] = acc[i][j];
        if (n0 == 0) out[(size_t)(m0 + i) * (K + 1) + K] = bias[i];
    }
}

// dtheta of one layer from the per-item partial sums (splits per item), in order (deterministic):
// n < K_s: weight W[m][n]; n == ldn - 1 (the row of ones): bias b[m].
__global__ void k_wgrad_reduce(LayerArgs la, const int32_t* __restrict__ item_start, int splits, int Mvalid, int ldn,
                               const float* __restrict__ part, float* __restrict__ dtheta)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)la.S * Mvalid * ldn) return;
    const int s = (int)(idx / ((int64_t)Mvalid * ldn));
    const int m = (int)((idx / ldn) % Mvalid);
    const int n = (int)(idx % ldn);
    const int K = la.K[s];
    if (m >= la.N[s] || (n >= K && n != ldn - 1)) return;
    float acc = 0.f;
    for (int it = item_start[s] * splits; it < item_start[s + 1] * splits; ++it)
        acc += part[((size_t)it * Mvalid + m) * ldn + n];
    if (n < K) dtheta[la.w_off[s] + (int64_t)m * K + n] = acc;
    else dtheta[la.b_off[s] + m] = acc;
}

// Stacked weights of layer l for all species (BF16 hi + lo or up to three TF32 parts):
//   fwd: out[(s*npad + n) * kpad + k] = W_s[n][k]      (n < n_out_s, k < n_in_s, else 0)
//   bwd: out[(s*npad + k) * kpad + n] = W_s[n][k]      (the transpose)
template <typename T>
__global__ void k_stack_weights(LayerArgs la, const float* __restrict__ theta, int npad, int kpad, int transpose,
                                T* __restrict__ out, T* __restrict__ out_lo, T* __restrict__ out_lo2,
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
    store_parts(out, out_lo, out_lo2, idx, v);
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

// 2D tensor [rows x cols] (row stride ld elements) of BF16 (box [box_rows x 64]) or FP32
// holding TF32 values (box [box_rows x 32]): 128-byte rows, 128 B swizzle
cudaError_t make_map(CUtensorMap* m, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows,
                     bool tf32 = false)
{
    const int64_t es = tf32 ? 4 : 2;
    if ((reinterpret_cast<uintptr_t>(base) & 15) || (ld * es) % 16) return cudaErrorInvalidValue;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)(rows > 0 ? rows : 1)};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * es)};
    cuuint32_t box[2] = {(cuuint32_t)(128 / es), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(m, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                          const_cast<void*>(base), dims, strides, box, estr,
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

template <int EPI, int PARTS, bool TF = false>
cudaError_t launch_tc_grid(const TcMaps& m, const TcArgs& ta, dim3 grid, cudaStream_t s)
{
    const int smem = (int)TcCfg<PARTS>::kSmem;
    cudaError_t e = cudaFuncSetAttribute(k_tc_gemm<EPI, PARTS, TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k_tc_gemm<EPI, PARTS, TF><<<grid, kTcThreads, smem, s>>>(m, ta);
    return cudaGetLastError();
}

// Persistent form of the row-tiled GEMM for the BF16 networks' layers (TC_FWD, TC_BWD_MID,
// TC_BWD_OUT).  One CTA per SM walks the work items (128-row tile of one species x N tile)
// with a stride of the grid size.  The TMA warp runs ahead through the stage ring across item
// boundaries; the MMA warp alternates between two TMEM accumulators, so the epilogue warps
// drain item j (tcgen05.ld, bias / activation, stores straight from registers: each thread
// writes whole 32-byte sectors of its own row) while the MMAs of item j + 1 run.  Barriers:
// full / empty per stage (TMA <-> MMA), acc_full / acc_empty per accumulator (MMA <->
// epilogue, the latter counting one arrival per epilogue warp).  Every wait is bounded.
__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

struct ItemPos {
    int s, row0, rend, n0;
    bool valid;
};

__device__ __forceinline__ ItemPos tc_item(const TcArgs& a, int item, int n_nt)
{
    ItemPos p;
    const int tile = item / n_nt, nt = item - tile * n_nt;
    int s = 0;
    while (tile >= a.tile_start[s + 1]) ++s;
    p.s = s;
    p.n0 = nt * a.BN;
    p.row0 = a.seg_off[s] + (tile - a.tile_start[s]) * kTcBM;
    p.rend = a.seg_off[s + 1];
    p.valid = p.n0 < a.N[s];
    return p;
}

template <int EPI, int PARTS>
__global__ void __launch_bounds__(kTcThreads, 1)
k_tc_gemm_p(const __grid_constant__ TcMaps tm, TcArgs a, int n_nt)
{
    using Cfg = TcCfg<PARTS>;
    constexpr int kStages = Cfg::kStages;
    constexpr int BKE = kTcBK;                           // BF16 elements per 128-byte K chunk
    constexpr int MMAK = 16;                             // K per instruction
    constexpr uint32_t kAcc = Cfg::kMaxBN;               // TMEM columns per accumulator
    extern __shared__ unsigned char smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;
    uint8_t* sB = smem + kStages * Cfg::kStageA;
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + kStages * Cfg::kStageB);
    uint64_t* empty = full + kStages;
    uint64_t* accf = empty + kStages;                    // [2]
    uint64_t* acce = accf + 2;                           // [2]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acce + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    // FP32 output staging, 2 KB per epilogue warp, past the barriers (kSmemP - kSmem bytes)
    float* stg = reinterpret_cast<float*>(sB + kStages * Cfg::kStageB + 256);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_items = a.tile_start[a.S] * n_nt;
    const int nk = (a.K + BKE - 1) / BKE;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) { mbar_init(full + i, 1); mbar_init(empty + i, 1); }
        for (int i = 0; i < 2; ++i) { mbar_init(accf + i, 1); mbar_init(acce + i, kTcEpiWarps); }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(tmem_slot, 2 * kAcc);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t bytes = Cfg::kParts * (kTileA + (uint32_t)a.BN * 128u);

    if (warp == 0) {
        if (lane == 0) {
            int g = 0;
            bool ok = true;
            for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
                const ItemPos ip = tc_item(a, item, n_nt);
                if (!ip.valid) continue;
                for (int kc = 0; kc < nk; ++kc, ++g) {
                    const int st = g % kStages;
                    const uint32_t ph = (uint32_t)(g / kStages) & 1u;
                    if (!mbar_wait(empty + st, ph ^ 1u, abort_flag)) { *abort_flag = 1; ok = false; break; }
                    mbar_expect_tx(full + st, bytes);
                    uint8_t* a_st = sA + st * Cfg::kStageA;
                    uint8_t* b_st = sB + st * Cfg::kStageB;
#pragma unroll
                    for (int q = 0; q < PARTS; ++q) {
                        tma_load_2d(a_st + q * kTileA, &tm.a[q], kc * BKE, ip.row0, full + st);
                        tma_load_2d(b_st + q * Cfg::kTileB, &tm.b[q], kc * BKE, ip.s * a.n_pad + ip.n0, full + st);
                    }
                }
            }
            // never leave with copies in flight
            for (int k = g > kStages ? g - kStages : 0; k < g; ++k)
                mbar_wait(full + k % kStages, (uint32_t)(k / kStages) & 1u, nullptr);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_mma(false, kTcBM, (uint32_t)a.BN);
            int g = 0, j = 0;
            bool ok = true;
            for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
                const ItemPos ip = tc_item(a, item, n_nt);
                if (!ip.valid) continue;
                const int b = j & 1;
                if (!mbar_wait(acce + b, ((uint32_t)(j >> 1) & 1u) ^ 1u, abort_flag)) { *abort_flag = 1; break; }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)b * kAcc;
                for (int kc = 0; kc < nk; ++kc, ++g) {
                    const int st = g % kStages;
                    const uint32_t ph = (uint32_t)(g / kStages) & 1u;
                    if (!mbar_wait(full + st, ph, abort_flag)) { *abort_flag = 1; ok = false; break; }
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(sA + st * Cfg::kStageA), b0 = smem_u32(sB + st * Cfg::kStageB);
#pragma unroll
                    for (int kk = 0; kk < BKE / MMAK; ++kk) {
                        const uint64_t a1 = sw128_desc(a0 + kk * 32), b1 = sw128_desc(b0 + kk * 32);
                        tc_mma<false>(d, a1, b1, idesc, (kc | kk) ? 1u : 0u);
                        if (PARTS >= 2) {
                            const uint64_t a2 = sw128_desc(a0 + kTileA + kk * 32);
                            const uint64_t b2 = sw128_desc(b0 + Cfg::kTileB + kk * 32);
                            tc_mma<false>(d, a1, b2, idesc, 1u);
                            tc_mma<false>(d, a2, b1, idesc, 1u);
                        }
                    }
                    tc_commit(empty + st);
                }
                tc_commit(accf + b);   // arrives once the item's MMAs have completed
                ++j;
            }
            // no TMEM release under running MMAs: the epilogue waited for every committed item;
            // after an abort wait (bounded) for whatever was issued last
            if (!ok || *abort_flag) {
                tc_commit(accf + (j & 1));
                mbar_wait(accf + (j & 1), ((uint32_t)(j >> 1) & 1u), nullptr);
            }
        }
    } else {
        const int ew = warp - 2;
        const int q = warp & 3;                    // TMEM lane quarter of this warp
        const int half = ew >> 2;
        int j = 0;
        for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
            const ItemPos ip = tc_item(a, item, n_nt);
            if (!ip.valid) continue;
            const int b = j & 1;
            const int r = ip.row0 + q * 32 + lane;
            const bool row_ok = r < ip.rend;
            const int s = ip.s, Ns = a.N[s];
            // BWD_MID: the pre-activations of the next 16 columns are loaded one chunk ahead (the
            // first before the wait for the MMAs), so their latency overlaps the TMEM wait and the
            // previous chunk's arithmetic and stores
            float zn[16];
            auto load_z = [&](int c) {
                const int n = ip.n0 + c;
                if (EPI != TC_BWD_MID || !row_ok || c >= a.BN || n >= Ns) return;
                const float* z = a.Zin + (size_t)r * a.ldZ + n;
                if (n + 16 <= Ns && (reinterpret_cast<uintptr_t>(z) & 15) == 0) {
#pragma unroll
                    for (int k = 0; k < 16; k += 4) {
                        const float4 t4 = *reinterpret_cast<const float4*>(z + k);
                        zn[k] = t4.x; zn[k + 1] = t4.y; zn[k + 2] = t4.z; zn[k + 3] = t4.w;
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < 16; ++k) zn[k] = (n + k < Ns) ? z[k] : 0.f;
                }
            };
            load_z(half * 16);
            if (!mbar_wait(accf + b, (uint32_t)(j >> 1) & 1u, abort_flag)) { *abort_flag = 1; break; }
            tc_fence_after();
            for (int c0 = half * 16; c0 < a.BN; c0 += 32) {
                float v[16];
                tc_ld16(tmem + (uint32_t)b * kAcc + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
                const int n = ip.n0 + c0;
                if (n >= Ns) continue;   // the same for the whole warp
                const bool whole = n + 16 <= Ns;
                float zv[16];
                if (EPI == TC_BWD_MID) {
#pragma unroll
                    for (int k = 0; k < 16; ++k) zv[k] = zn[k];
                    load_z(c0 + 32);
                }
                float o1[16], o2[16];
                if (EPI == TC_FWD) {
                    const float* bias = a.bias + s * a.n_pad + n;
                    float bv[16];
                    if ((reinterpret_cast<uintptr_t>(bias) & 15) == 0) {
#pragma unroll
                        for (int k = 0; k < 16; k += 4) {
                            const float4 t4 = *reinterpret_cast<const float4*>(bias + k);
                            bv[k] = t4.x; bv[k + 1] = t4.y; bv[k + 2] = t4.z; bv[k + 3] = t4.w;
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < 16; ++k) bv[k] = bias[k];
                    }
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        o1[k] = v[k] + bv[k];
                        o2[k] = act_f(a.act[s], o1[k]);
                    }
                } else if (EPI == TC_BWD_MID) {
#pragma unroll
                    for (int k = 0; k < 16; ++k) o2[k] = (whole || n + k < Ns) ? v[k] * act_d1(a.act[s], zv[k]) : 0.f;
                } else {
#pragma unroll
                    for (int k = 0; k < 16; ++k) o1[k] = v[k];
                }
                if (EPI == TC_FWD || EPI == TC_BWD_OUT) {
                    const bool aligned = (a.ldF & 3) == 0 &&
                                         (reinterpret_cast<uintptr_t>(a.outF + (size_t)ip.row0 * a.ldF + n) & 15) == 0;
                    if (whole && aligned) {
                        // through the warp's staging tile: each lane writes its row's 16 values
                        // (16-byte pieces swizzled by row, conflict-free), then the warp stores
                        // 8 rows x 64 contiguous bytes per instruction instead of 32 rows x 16
                        float* st = stg + ew * 512;
                        const int sw = (lane >> 1) & 3;
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            *reinterpret_cast<float4*>(st + lane * 16 + 4 * (k ^ sw)) =
                                make_float4(o1[4 * k], o1[4 * k + 1], o1[4 * k + 2], o1[4 * k + 3]);
                        __syncwarp();
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int row = i * 8 + (lane >> 2), pc = lane & 3;
                            const float4 val = *reinterpret_cast<const float4*>(st + row * 16 + 4 * (pc ^ ((row >> 1) & 3)));
                            const int rr = ip.row0 + q * 32 + row;
                            if (rr < ip.rend)
                                *reinterpret_cast<float4*>(a.outF + (size_t)rr * a.ldF + n + 4 * pc) = val;
                        }
                        __syncwarp();
                    } else if (row_ok) {
                        float* o = a.outF + (size_t)r * a.ldF + n;
#pragma unroll
                        for (int k = 0; k < 16; ++k)
                            if (n + k < Ns) o[k] = o1[k];
                    }
                }
                if (EPI == TC_FWD || EPI == TC_BWD_MID) {
                    const bool aligned = (a.ldH & 7) == 0 &&
                                         (reinterpret_cast<uintptr_t>(a.outH + (size_t)ip.row0 * a.ldH + n) & 15) == 0 &&
                                         (PARTS < 2 ||
                                          (reinterpret_cast<uintptr_t>(a.outL + (size_t)ip.row0 * a.ldH + n) & 15) == 0);
                    if (whole && aligned) {
                        uint32_t hw[8], lw[8];
#pragma unroll
                        for (int k = 0; k < 16; k += 2) {
                            const __nv_bfloat16 h0 = __float2bfloat16_rn(o2[k]), h1 = __float2bfloat16_rn(o2[k + 1]);
                            const __nv_bfloat16 l0 = __float2bfloat16_rn(o2[k] - __bfloat162float(h0));
                            const __nv_bfloat16 l1 = __float2bfloat16_rn(o2[k + 1] - __bfloat162float(h1));
                            hw[k / 2] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                            lw[k / 2] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
                        }
                        // through the staging tile: hi rows then lo rows, 32 B per row, the two
                        // 16-byte pieces swapped on every other group of four rows (conflict-free);
                        // the warp then stores 16 rows x 32 contiguous bytes per instruction
                        uint4* st = reinterpret_cast<uint4*>(stg + ew * 512);
                        const int sw = (lane >> 2) & 1;
                        st[lane * 2 + (0 ^ sw)] = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                        st[lane * 2 + (1 ^ sw)] = make_uint4(hw[4], hw[5], hw[6], hw[7]);
                        if (PARTS >= 2) {
                            st[64 + lane * 2 + (0 ^ sw)] = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                            st[64 + lane * 2 + (1 ^ sw)] = make_uint4(lw[4], lw[5], lw[6], lw[7]);
                        }
                        __syncwarp();
#pragma unroll
                        for (int part = 0; part < (PARTS >= 2 ? 2 : 1); ++part) {
                            __nv_bfloat16* base = part ? a.outL : a.outH;
#pragma unroll
                            for (int i = 0; i < 2; ++i) {
                                const int row = i * 16 + (lane >> 1), pc = lane & 1;
                                const uint4 val = st[part * 64 + row * 2 + (pc ^ ((row >> 2) & 1))];
                                const int rr = ip.row0 + q * 32 + row;
                                if (rr < ip.rend)
                                    *reinterpret_cast<uint4*>(base + (size_t)rr * a.ldH + n + 8 * pc) = val;
                            }
                        }
                        __syncwarp();
                    } else if (row_ok) {
#pragma unroll
                        for (int k = 0; k < 16; ++k)
                            if (n + k < Ns)
                                store_split(a.outH, PARTS >= 2 ? a.outL : nullptr, (size_t)r * a.ldH + n + k, o2[k]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acce + b);
            ++j;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) set_status(a.status, PANNA_ERR_TIMEOUT, blockIdx.x);
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, 2 * kAcc);
    }
}

// row-tiled launch: one CTA per (species, 128-row tile) and N tile
template <int EPI, int PARTS, bool TF = false>
cudaError_t launch_tc(const TcMaps& m, const TcArgs& ta, int64_t N, int nmax, cudaStream_t s)
{
    dim3 grid((unsigned)((N + kTcBM - 1) / kTcBM + ta.S), (unsigned)((nmax + ta.BN - 1) / ta.BN));
    return launch_tc_grid<EPI, PARTS, TF>(m, ta, grid, s);
}

// persistent launch: one CTA per SM (at most one per work item)
template <int EPI, int PARTS>
cudaError_t launch_tc_p(const TcMaps& m, const TcArgs& ta, int64_t N, int nmax, cudaStream_t s)
{
    static int n_sm = 0;
    if (n_sm == 0) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
    }
    const int n_nt = (nmax + ta.BN - 1) / ta.BN;
    const int64_t items = ((N + kTcBM - 1) / kTcBM + ta.S) * n_nt;
    const unsigned grid = (unsigned)std::min<int64_t>(items, n_sm);
    const int smem = (int)TcCfg<PARTS>::kSmemP;
    cudaError_t e = cudaFuncSetAttribute(k_tc_gemm_p<EPI, PARTS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k_tc_gemm_p<EPI, PARTS><<<grid, kTcThreads, smem, s>>>(m, ta, n_nt);
    return cudaGetLastError();
}

template <int EPI>
cudaError_t launch_tc_any(bool split, const TcMaps& m, const TcArgs& ta, int64_t N, int nmax, cudaStream_t s)
{
    return split ? launch_tc_p<EPI, 2>(m, ta, N, nmax, s) : launch_tc_p<EPI, 1>(m, ta, N, nmax, s);
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
    const int max_bn = split ? TcCfg<2>::kMaxBN : TcCfg<1>::kMaxBN;
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
void tc_g16(const MlpPlan& p, int64_t N, bool split, void* ws, __nv_bfloat16** hi, __nv_bfloat16** lo)
{
    TcBufs t;
    tc_carve(p, N, split, static_cast<char*>(ws), t);
    *hi = t.ldh[0] == p.ld[0] ? t.G16[0] : nullptr;
    *lo = t.ldh[0] == p.ld[0] ? t.G16[1] : nullptr;
}

cudaError_t mlp_bf16_energy_grad(const MlpPlan& p, const MlpBuffers& b, const float* theta, int64_t N, void* ws,
                                 bool split, float* E_rows, float* g, DevStatus* status, cudaStream_t s,
                                 int* launches, bool g16_ready)
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
        k_stack_weights<__nv_bfloat16><<<(unsigned)((tf + 255) / 256), 256, 0, s>>>(la, theta, t.npf[l], round_up(ni, 8), 0,
                                                                    t.Wf[l][0], t.Wf[l][1], nullptr, t.bias[l]);
        int64_t tb = (int64_t)p.S * t.npb[l] * round_up(no, 8);
        k_stack_weights<__nv_bfloat16><<<(unsigned)((tb + 255) / 256), 256, 0, s>>>(la, theta, t.npb[l], round_up(no, 8), 1,
                                                                    t.Wb[l][0], t.Wb[l][1], nullptr, nullptr);
        *launches += 2;
    }
    // padding columns of the BF16 operands meet zero weights, but must not hold NaN (the
    // epilogues write the species' own columns only); layers without padding need no clearing
    for (int l = 1; l < p.L; ++l) {
        bool pad = false;
        for (int q = 0; q < p.S; ++q) pad = pad || p.widths[q][l] != t.ldh[l];
        if (!pad) continue;
        for (int q = 0; q < parts; ++q) {
            e = cudaMemsetAsync(t.A16[l][q], 0, (size_t)N * t.ldh[l] * 2, s);
            if (e == cudaSuccess) e = cudaMemsetAsync(t.Zb16[l][q], 0, (size_t)N * t.ldh[l] * 2, s);
            if (e != cudaSuccess) return e;
        }
    }
    if (!g16_ready) {
        k_to_bf16<<<(unsigned)((N * t.ldh[0] + 255) / 256), 256, 0, s>>>(N * t.ldh[0], b.G, t.G16[0], t.G16[1]);
        ++*launches;
    }

    TcArgs base{};
    base.S = p.S;
    base.seg_off = b.seg_off;
    base.tile_start = t.tiles128;
    base.status = status;
    TcMaps maps;
    // forward through the hidden layers
    for (int l = 0; l < p.L - 1; ++l) {
        CUtensorMap mA[2], mB[2];
        __nv_bfloat16* const* Ain = l == 0 ? t.G16 : t.A16[l];
        e = make_maps(mA, Ain, parts, N, p.ld[l], t.ldh[l], kTcBM);
        if (e == cudaSuccess)
            e = make_maps(mB, t.Wf[l], parts, (int64_t)p.S * t.npf[l], p.ld[l], round_up(p.ld[l], 8), t.bnf[l]);
        if (e != cudaSuccess) return e;
        maps.a[0] = mA[0]; maps.b[0] = mB[0]; maps.a[1] = mA[1]; maps.b[1] = mB[1];
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
        maps.a[0] = mA[0]; maps.b[0] = mB[0]; maps.a[1] = mA[1]; maps.b[1] = mB[1];
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

// ------------------------------------------------------------------ FP32 networks, first layer on TF32 pairs
//
// The first layer (descriptor width D -> first hidden width) carries almost all of the
// networks' arithmetic.  With FP32 networks it runs on the tensor cores as TF32 hi + lo
// pairs (three MMAs per product, about 22 significant bits per operand); the narrow deeper
// layers stay on the CUDA-core kernels of mlp.cu.

namespace {

// Parts per operand: three (exact splits of FP32, products exact to 2^-32) for the forward
// and input-gradient products, two in the training-only products (tangent, weight
// gradient).  The accumulation inside the MMA, not the operand split, then limits the
// accuracy: its error grows with the length of the K chain about linearly (a CUDA-core
// FP32 chain rounds to nearest and grows about as its square root), so the forward
// product, whose error reaches the forces through act' and act'', stays on the CUDA cores
// unless TF32_FWD is asked for.
constexpr int kPartsFwd = 3, kPartsTan = 2, kPartsW = 2;

struct Tf32Bufs {
    int32_t* tiles128;
    int32_t* pstart;
    int32_t* items;
    float* Wf[3];          // [S * npf, kpf]   W_1, K-major over D
    float* Wb[3];          // [S * npb, kpb]   W_1^T, K-major over the first hidden width
    float* bias;           // [S * npf]
    float* G[3];           // [N, D]           descriptors (forward), then their tangent (training)
    float* Zb[3];          // [N, ldz]         zbar_1 of the input gradient
    float* ZT[3];          // [max width, 2 Kp]  zbar_l | zdotbar_l, atoms along columns (2 parts)
    float* GT[3];          // [max input + 1, 2 Kp]  A_{l-1} (+ a row of ones) | Adot_{l-1}, likewise
    float* part;           // [items, max over layers of ld[l+1] (ld[l] + 1)]
    int npf, npb, bnf, bnb, bnw, kpf, kpb, ldz, chunk, items_max;
    int64_t Kp;
};

// buffers of the products in `mask` (TF32_* bits) only
size_t tf32_carve(const MlpPlan& p, int64_t N, int mask, char* base, Tf32Bufs& t)
{
    size_t off = 0;
    auto take = [&](size_t n) {
        void* q = base ? base + off : nullptr;
        off += (n + 255) & ~(size_t)255;
        return q;
    };
    const int D = p.ld[0], h1 = p.ld[1], S = p.S;
    const int maxbn = TcCfg<kPartsFwd>::kMaxBN;
    t.bnf = tc_bn(h1, maxbn); t.npf = round_up(h1, t.bnf); t.kpf = round_up(D, 4);
    t.bnb = tc_bn(D, maxbn); t.npb = round_up(D, t.bnb); t.kpb = round_up(h1, 4);
    t.bnw = tc_bn(D + 1, TcCfg<kPartsW>::kMaxBN);
    t.ldz = round_up(h1, 4);
    t.Kp = (N + 31) / 32 * 32 + 32 * (int64_t)S;
    t.chunk = (int)std::max<int64_t>(512, (N / 256 + 31) / 32 * 32);
    t.items_max = (int)((t.Kp + t.chunk - 1) / t.chunk) + S;
    t.tiles128 = static_cast<int32_t*>(take((kMaxSpecies + 1) * sizeof(int32_t)));
    t.pstart = static_cast<int32_t*>(take((kMaxSpecies + 1) * sizeof(int32_t)));
    t.items = static_cast<int32_t*>(take((kMaxSpecies + 1) * sizeof(int32_t)));
    const int pf = (mask & TF32_FWD) ? kPartsFwd : ((mask & TF32_TAN) ? kPartsTan : 0);   // W_1 and G parts
    const int pb = (mask & TF32_INGRAD) ? kPartsFwd : 0;
    const int pw = (mask & TF32_WGRAD) ? kPartsW : 0;
    int in_max = 0;   // widest layer input (rows of the transposed inputs, plus the row of ones)
    for (int l = 0; l < p.L; ++l) in_max = std::max(in_max, p.ld[l]);
    for (int q = 0; q < 3; ++q) {
        t.Wf[q] = q < pf ? static_cast<float*>(take((size_t)S * t.npf * t.kpf * 4)) : nullptr;
        t.G[q] = q < pf ? static_cast<float*>(take((size_t)N * D * 4)) : nullptr;
        t.Wb[q] = q < pb ? static_cast<float*>(take((size_t)S * t.npb * t.kpb * 4)) : nullptr;
        t.Zb[q] = q < pb ? static_cast<float*>(take((size_t)N * t.ldz * 4)) : nullptr;
        t.ZT[q] = q < pw ? static_cast<float*>(take((size_t)p.max_hidden * 2 * t.Kp * 4)) : nullptr;
        t.GT[q] = q < pw ? static_cast<float*>(take((size_t)(in_max + 1) * 2 * t.Kp * 4)) : nullptr;
    }
    t.bias = static_cast<float*>(take((size_t)S * t.npf * 4));
    size_t part_max = 0;
    for (int l = 0; l < p.L; ++l) part_max = std::max(part_max, (size_t)p.ld[l + 1] * (p.ld[l] + 1));
    t.part = pw ? static_cast<float*>(take((size_t)t.items_max * part_max * 4)) : nullptr;
    return off + 4096;
}

Parts3 parts_of(float* const* b, int parts)
{
    Parts3 o{};
    for (int q = 0; q < parts; ++q) o.p[q] = b[q];
    return o;
}

cudaError_t tf32_maps(TcMaps& m, int parts, float* const* a, int64_t arows, int64_t acols, int64_t alda, int abox,
                      float* const* b, int64_t brows, int64_t bcols, int64_t bldb, int bbox)
{
    for (int q = 0; q < parts; ++q) {
        cudaError_t e = make_map(&m.a[q], a[q], arows, acols, alda, abox, true);
        if (e == cudaSuccess) e = make_map(&m.b[q], b[q], brows, bcols, bldb, bbox, true);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

TcArgs tf32_base(const MlpPlan& p, const MlpBuffers& b, const Tf32Bufs& t, DevStatus* status)
{
    TcArgs ta{};
    ta.S = p.S;
    ta.seg_off = b.seg_off;
    ta.tile_start = t.tiles128;
    ta.status = status;
    return ta;
}

unsigned blocks(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

bool tf32_first_layer_ok(const MlpPlan& p) { return p.L >= 2 && p.ld[0] % 4 == 0; }

size_t tf32_workspace_bytes(const MlpPlan& p, int64_t N, int mask)
{
    Tf32Bufs t;
    return tf32_carve(p, N, mask, nullptr, t);
}

cudaError_t tf32_prepare(const MlpPlan& p, const MlpBuffers& b, const float* theta, int64_t N, void* ws, int mask,
                         cudaStream_t s, int* launches)
{
    cudaError_t e = get_encoder();
    if (e != cudaSuccess) return e;
    Tf32Bufs t;
    tf32_carve(p, N, mask, static_cast<char*>(ws), t);
    k_tiles128<<<1, 32, 0, s>>>(p.S, b.seg_off, t.tiles128);
    ++*launches;
    LayerArgs la = tc_layer_args(p, 0);
    if (t.Wf[0]) {
        k_stack_weights<float><<<blocks((int64_t)p.S * t.npf * t.kpf), 256, 0, s>>>(la, theta, t.npf, t.kpf, 0, t.Wf[0],
                                                                                   t.Wf[1], t.Wf[2], t.bias);
        ++*launches;
    }
    if (t.Wb[0]) {
        k_stack_weights<float><<<blocks((int64_t)p.S * t.npb * t.kpb), 256, 0, s>>>(la, theta, t.npb, t.kpb, 1, t.Wb[0],
                                                                                   t.Wb[1], t.Wb[2], nullptr);
        ++*launches;
    }
    if (mask & TF32_WGRAD) {
        k_tf32_items<<<1, 32, 0, s>>>(p.S, b.seg_off, t.chunk, t.pstart, t.items);
        ++*launches;
    }
    return cudaGetLastError();
}

// Z_1 = G W_1^T + b_1, A_1 = act(Z_1) (FP32 out)
cudaError_t tf32_forward1(const MlpPlan& p, const MlpBuffers& b, int64_t N, void* ws, int mask, DevStatus* status,
                          cudaStream_t s, int* launches)
{
    Tf32Bufs t;
    tf32_carve(p, N, mask, static_cast<char*>(ws), t);
    const int D = p.ld[0];
    k_split_tf32<<<blocks(N * D), 256, 0, s>>>(N, D, D, D, b.G, parts_of(t.G, kPartsFwd));
    ++*launches;
    TcMaps m;
    cudaError_t e = tf32_maps(m, kPartsFwd, t.G, N, D, D, kTcBM, t.Wf, (int64_t)p.S * t.npf, D, t.kpf, t.bnf);
    if (e != cudaSuccess) return e;
    TcArgs ta = tf32_base(p, b, t, status);
    for (int q = 0; q < p.S; ++q) { ta.N[q] = p.widths[q][1]; ta.act[q] = p.acts[q][0]; }
    ta.K = D; ta.BN = t.bnf; ta.n_pad = t.npf; ta.bias = t.bias;
    ta.outF = b.Z[1]; ta.ldF = p.ld[1];
    ta.outA = b.A[1]; ta.ldA = p.ld[1];
    e = launch_tc<TC_FWD32, kPartsFwd, true>(m, ta, N, p.ld[1], s);
    ++*launches;
    return e;
}

// tangent of the first layer along Gdot: Zd_1 = Gdot W_1^T, Ad_1 = act'(Z_1) Zd_1
cudaError_t tf32_tangent1(const MlpPlan& p, const MlpBuffers& b, int64_t N, void* ws, int mask, const float* Gdot,
                          DevStatus* status, cudaStream_t s, int* launches)
{
    Tf32Bufs t;
    tf32_carve(p, N, mask, static_cast<char*>(ws), t);
    const int D = p.ld[0];
    // the forward pass is done with its split of G: the buffers now take Gdot
    k_split_tf32<<<blocks(N * D), 256, 0, s>>>(N, D, D, D, Gdot, parts_of(t.G, kPartsTan));
    ++*launches;
    TcMaps m;
    cudaError_t e = tf32_maps(m, kPartsTan, t.G, N, D, D, kTcBM, t.Wf, (int64_t)p.S * t.npf, D, t.kpf, t.bnf);
    if (e != cudaSuccess) return e;
    TcArgs ta = tf32_base(p, b, t, status);
    for (int q = 0; q < p.S; ++q) { ta.N[q] = p.widths[q][1]; ta.act[q] = p.acts[q][0]; }
    ta.K = D; ta.BN = t.bnf; ta.n_pad = t.npf;
    ta.outF = b.Zd[1]; ta.ldF = p.ld[1];
    ta.outA = b.Ad[1]; ta.ldA = p.ld[1];
    ta.Zin = b.Z[1]; ta.ldZ = p.ld[1];
    e = launch_tc<TC_TAN32, kPartsTan, true>(m, ta, N, p.ld[1], s);
    ++*launches;
    return e;
}

// Weight gradient of layer l+1 (l = 0: the first layer, inputs G and Gdot):
//   dW = Zb^T A_l + Zdb^T Adot_l,  db = sum of Zb over the species' atoms,
// sums over atoms on the tensor cores (TF32 pairs), written into dtheta.  Zb, Zdb: the
// layer's adjoints [N, ld[l+1]]; A, Ad: its inputs [N, ld[l]].
cudaError_t tf32_wgrad(const MlpPlan& p, const MlpBuffers& b, int64_t N, void* ws, int mask, int l, const float* A,
                       const float* Ad, float* dtheta, DevStatus* status, cudaStream_t s, int* launches)
{
    Tf32Bufs t;
    tf32_carve(p, N, mask, static_cast<char*>(ws), t);
    const int K = p.ld[l], M = p.ld[l + 1];
    LayerArgs la = tc_layer_args(p, l);
    const int O = M * (K + 1);
    if (l > 0 && O <= 256 * kSmallOut && M + K <= 192) {
        // narrow layer: CUDA cores, no transposed copies (row staging <= 48 KB of shared memory)
        size_t part_max = 0;
        for (int q = 0; q < p.L; ++q) part_max = std::max(part_max, (size_t)p.ld[q + 1] * (p.ld[q] + 1));
        const int splits = (int)std::max<size_t>(1, std::min<size_t>(8, part_max / O));
        const size_t smem = (size_t)kSmallRows * 2 * (M + K) * sizeof(float);
        dim3 grid((unsigned)t.items_max, (unsigned)splits);
        if (M % 4 == 0 && K % 4 == 0 && (M / 4) * (K / 4) <= 256)
            k_wgrad_small4<<<grid, 256, smem, s>>>(p.S, b.seg_off, t.items, t.chunk, splits, M, K, b.Zb, b.Zdb, A,
                                                  Ad, t.part);
        else
            k_wgrad_small<<<grid, 256, smem, s>>>(p.S, b.seg_off, t.items, t.chunk, splits, M, K, b.Zb, b.Zdb, A, Ad,
                                                 t.part);
        k_wgrad_reduce<<<blocks((int64_t)p.S * O), 256, 0, s>>>(la, t.items, splits, M, K + 1, t.part, dtheta);
        *launches += 2;
        return cudaGetLastError();
    }
    const int64_t ldT = 2 * t.Kp;
    Widths wz{}, wg{};
    for (int q = 0; q < p.S; ++q) { wz.n[q] = p.widths[q][l + 1]; wg.n[q] = p.widths[q][l]; }
    const unsigned ctiles = (unsigned)(t.Kp / 32);
    const Parts3 zt = parts_of(t.ZT, kPartsW), gt = parts_of(t.GT, kPartsW);
    k_transpose_split<<<dim3(ctiles, (unsigned)((M + 31) / 32)), 256, 0, s>>>(
        b.Zb, M, p.S, b.seg_off, t.pstart, wz, M, -1, zt, ldT, 0);
    k_transpose_split<<<dim3(ctiles, (unsigned)((M + 31) / 32)), 256, 0, s>>>(
        b.Zdb, M, p.S, b.seg_off, t.pstart, wz, M, -1, zt, ldT, t.Kp);
    k_transpose_split<<<dim3(ctiles, (unsigned)((K + 1 + 31) / 32)), 256, 0, s>>>(
        A, K, p.S, b.seg_off, t.pstart, wg, K + 1, K, gt, ldT, 0);
    k_transpose_split<<<dim3(ctiles, (unsigned)((K + 1 + 31) / 32)), 256, 0, s>>>(
        Ad, K, p.S, b.seg_off, t.pstart, wg, K + 1, -1, gt, ldT, t.Kp);
    *launches += 4;
    const int bn = tc_bn(K + 1, TcCfg<kPartsW>::kMaxBN);
    TcMaps m;
    cudaError_t e = tf32_maps(m, kPartsW, t.ZT, M, ldT, ldT, kTcBM, t.GT, K + 1, ldT, ldT, bn);
    if (e != cudaSuccess) return e;
    TcArgs ta = tf32_base(p, b, t, status);
    ta.BN = bn;
    ta.item_start = t.items; ta.pstart = t.pstart; ta.Kp = (int)t.Kp; ta.chunk = t.chunk;
    ta.part = t.part; ta.ldn = K + 1; ta.Mvalid = M; ta.Nvalid = K + 1;
    dim3 grid((unsigned)t.items_max, (unsigned)((K + 1 + bn - 1) / bn), (unsigned)((M + kTcBM - 1) / kTcBM));
    e = launch_tc_grid<TC_WGRAD, kPartsW, true>(m, ta, grid, s);
    if (e != cudaSuccess) return e;
    k_wgrad_reduce<<<blocks((int64_t)p.S * M * (K + 1)), 256, 0, s>>>(la, t.items, 1, M, K + 1, t.part, dtheta);
    *launches += 2;
    return cudaGetLastError();
}

}  // namespace panna
