// Cell-list neighbour search on the GPU (locality within rc, Sec. I / Sec. II.A).
//
// Stages, all on the caller's stream:
//   k_cfg_geom     one warp per configuration: frame, fractional bounding box, cell grid
//                  (cells at least rc wide), image-shift table;
//   k_bin          one thread per atom: fold into the cell, split the folded FP64
//                  position into FP32 hi + lo, count atoms per cell;
//   scan           exclusive scan of the cell counts;
//   k_scatter / k_sort_cells   atoms of each cell, sorted by index (deterministic);
//   k_neighbors    one warp per atom: scan the 3x3x3 (or wider) block of cells, FP32
//                  filter on hi parts, then the relative vector in double-float (FP32
//                  hi + lo, error-free sums) and an FP64 re-test for the rare pairs whose
//                  squared distance lies within 2e-6 rc^2 of the cutoff -- so the
//                  neighbour set equals the FP64 definition for inputs with no pair within
//                  1e-6 A of rc; entries are stored grouped by neighbour species.
//   k_species_*    stable counting sort of atoms by species (network row order).
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace panna {

// ------------------------------------------------------------------ scan (int64)

constexpr int kScanThreads = 256;
constexpr int kScanPer = 4;
constexpr int kScanTile = kScanThreads * kScanPer;

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// exclusive scan of one value per thread over a 256-thread block; returns the block total
__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t& excl)
{
    __shared__ int64_t wsum[kScanThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t inc = warp_incl_scan(v);
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int64_t s = lane < kScanThreads / 32 ? wsum[lane] : 0;
        s = warp_incl_scan(s);
        if (lane < kScanThreads / 32) wsum[lane] = s;
    }
    __syncthreads();
    int64_t before = wid > 0 ? wsum[wid - 1] : 0;
    excl = before + inc - v;
    int64_t total = wsum[kScanThreads / 32 - 1];
    __syncthreads();
    return total;
}

__global__ void k_scan_reduce(const int64_t* __restrict__ in, int64_t n, int64_t* __restrict__ sums)
{
    int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanPer;
    int64_t v = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k)
        if (base + k < n) v += in[base + k];
    int64_t ex;
    int64_t tot = block_excl_scan(v, ex);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan_sums(int64_t* sums, int64_t nb)
{
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < nb; b0 += kScanThreads) {
        int64_t k = b0 + threadIdx.x;
        int64_t v = k < nb ? sums[k] : 0;
        int64_t ex;
        int64_t tot = block_excl_scan(v, ex);
        if (k < nb) sums[k] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[nb] = carry;
}

__global__ void k_scan_final(const int64_t* __restrict__ in, int64_t* __restrict__ out, int64_t n,
                             const int64_t* __restrict__ sums)
{
    int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanPer;
    int64_t v[kScanPer];
    int64_t t = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        v[k] = base + k < n ? in[base + k] : 0;
        t += v[k];
    }
    int64_t ex;
    block_excl_scan(t, ex);
    int64_t run = sums[blockIdx.x] + ex;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = sums[gridDim.x];
}

int64_t scan_scratch_elems(int64_t n) { return (n + kScanTile - 1) / kScanTile + 2; }

cudaError_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* tmp, cudaStream_t s,
                               int* launches)
{
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb == 0) nb = 1;
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, tmp);
    k_scan_sums<<<1, kScanThreads, 0, s>>>(tmp, nb);
    k_scan_final<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, tmp);
    *launches += 3;
    return cudaGetLastError();
}

// ------------------------------------------------------------------ geometry per config

__device__ __forceinline__ int atom_config(const int64_t* __restrict__ off, int64_t C, int64_t i)
{
    int64_t lo = 0, hi = C - 1;  // largest c with off[c] <= i
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return (int)lo;
}

__global__ void k_atom_cfg(const int64_t* __restrict__ off, int64_t C, int64_t N, int32_t* __restrict__ atom_cfg)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) atom_cfg[i] = atom_config(off, C, i);
}

// One warp per configuration (kCfgWarps per block).
constexpr int kCfgWarps = 8;

__device__ __forceinline__ double warp_min_d(double v)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_max_d(double v)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__global__ void __launch_bounds__(kCfgWarps * 32)
k_cfg_geom(panna_system sys, double rc, CfgGeom* __restrict__ geom, int64_t* __restrict__ cfg_cells, DevStatus* st)
{
    const int lane = threadIdx.x & 31;
    const int64_t c = (int64_t)blockIdx.x * kCfgWarps + (threadIdx.x >> 5);
    if (c >= sys.n_cfg) return;
    const int64_t a0 = sys.atom_off[c], a1 = sys.atom_off[c + 1];
    int per[3];
    for (int a = 0; a < 3; ++a) per[a] = sys.pbc[3 * c + a] ? 1 : 0;
    const bool any = per[0] || per[1] || per[2];
    double frame[9], finv[9];
    for (int k = 0; k < 9; ++k) frame[k] = finv[k] = (k % 4 == 0 ? 1.0 : 0.0);
    if (any) {
        for (int k = 0; k < 9; ++k) frame[k] = sys.cell[9 * c + k];
        const double* m = frame;
        double det = m[0] * (m[4] * m[8] - m[5] * m[7]) - m[1] * (m[3] * m[8] - m[5] * m[6])
                   + m[2] * (m[3] * m[7] - m[4] * m[6]);
        if (!(fabs(det) > 1e-12) || !isfinite(det)) {
            if (lane == 0) set_status(st, PANNA_ERR_BAD_INPUT, (int)c);
            for (int k = 0; k < 9; ++k) frame[k] = (k % 4 == 0 ? 1.0 : 0.0);
            per[0] = per[1] = per[2] = 0;
        } else {
            const double id = 1.0 / det;
            finv[0] = (m[4] * m[8] - m[5] * m[7]) * id;
            finv[1] = (m[2] * m[7] - m[1] * m[8]) * id;
            finv[2] = (m[1] * m[5] - m[2] * m[4]) * id;
            finv[3] = (m[5] * m[6] - m[3] * m[8]) * id;
            finv[4] = (m[0] * m[8] - m[2] * m[6]) * id;
            finv[5] = (m[2] * m[3] - m[0] * m[5]) * id;
            finv[6] = (m[3] * m[7] - m[4] * m[6]) * id;
            finv[7] = (m[1] * m[6] - m[0] * m[7]) * id;
            finv[8] = (m[0] * m[4] - m[1] * m[3]) * id;
        }
    }
    // fractional bounding box (needed on non-periodic directions only)
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    if (!(per[0] && per[1] && per[2])) {
        for (int64_t i = a0 + lane; i < a1; i += 32) {
            const double* x = sys.pos + 3 * i;
            for (int a = 0; a < 3; ++a) {
                double sa = x[0] * finv[a] + x[1] * finv[3 + a] + x[2] * finv[6 + a];
                lo[a] = fmin(lo[a], sa);
                hi[a] = fmax(hi[a], sa);
            }
        }
        for (int a = 0; a < 3; ++a) { lo[a] = warp_min_d(lo[a]); hi[a] = warp_max_d(hi[a]); }
    }
    CfgGeom& g = geom[c];
    // image shift table for t in [-1,1]^3, one entry per lane
    if (lane < 27) {
        const int t0 = lane / 9 - 1, t1 = (lane / 3) % 3 - 1, t2 = lane % 3 - 1;
        for (int d = 0; d < 3; ++d) {
            double S = t0 * frame[d] + t1 * frame[3 + d] + t2 * frame[6 + d];
            float sh = (float)S;
            g.sh_hi[lane][d] = sh;
            g.sh_lo[lane][d] = (float)(S - (double)sh);
        }
    }
    if (lane != 0) return;
    for (int k = 0; k < 9; ++k) { g.cell[k] = frame[k]; g.cinv[k] = finv[k]; }
    // perpendicular widths of the frame
    const double* A = frame; const double* B = frame + 3; const double* Cc = frame + 6;
    double bxc[3] = {B[1] * Cc[2] - B[2] * Cc[1], B[2] * Cc[0] - B[0] * Cc[2], B[0] * Cc[1] - B[1] * Cc[0]};
    double cxa[3] = {Cc[1] * A[2] - Cc[2] * A[1], Cc[2] * A[0] - Cc[0] * A[2], Cc[0] * A[1] - Cc[1] * A[0]};
    double axb[3] = {A[1] * B[2] - A[2] * B[1], A[2] * B[0] - A[0] * B[2], A[0] * B[1] - A[1] * B[0]};
    double vol = fabs(A[0] * bxc[0] + A[1] * bxc[1] + A[2] * bxc[2]);
    double h[3] = {vol / sqrt(bxc[0] * bxc[0] + bxc[1] * bxc[1] + bxc[2] * bxc[2]),
                   vol / sqrt(cxa[0] * cxa[0] + cxa[1] * cxa[1] + cxa[2] * cxa[2]),
                   vol / sqrt(axb[0] * axb[0] + axb[1] * axb[1] + axb[2] * axb[2])};
    const double rcw = rc * (1.0 + 1e-9);   // cells strictly wider than rc
    double ext[3];
    const int64_t n_at = a1 - a0;
    for (int a = 0; a < 3; ++a) {
        g.per[a] = per[a];
        if (per[a]) {
            g.lo[a] = 0.0;
            ext[a] = 1.0;
        } else {
            g.lo[a] = n_at > 0 ? lo[a] : 0.0;
            ext[a] = n_at > 0 ? fmax(hi[a] - lo[a], 0.0) : 0.0;
        }
        double nc = floor(ext[a] * h[a] / rcw);
        g.n[a] = nc < 1.0 ? 1 : (nc > 1024.0 ? 1024 : (int)nc);
    }
    // no more cells than max(1, 2 * atoms): wider cells keep the search exact
    const int64_t lim = n_at > 0 ? 2 * n_at : 1;
    while ((int64_t)g.n[0] * g.n[1] * g.n[2] > lim) {
        int a = 0;
        if (g.n[1] > g.n[a]) a = 1;
        if (g.n[2] > g.n[a]) a = 2;
        g.n[a] = (g.n[a] + 1) / 2;
    }
    for (int a = 0; a < 3; ++a) {
        const double e = ext[a] > 0.0 ? ext[a] : 1.0;
        g.inv_w[a] = (double)g.n[a] / e;
        const double cw = h[a] * e / g.n[a];   // perpendicular cell width
        int K = 1;
        if (per[a] && cw < rcw) K = (int)ceil(rcw / cw);
        g.K[a] = K;
    }
    g.ncells = g.n[0] * g.n[1] * g.n[2];
    g.cell_base = 0;
    cfg_cells[c] = g.ncells;
}

__global__ void k_set_cell_base(CfgGeom* __restrict__ geom, const int64_t* __restrict__ base, int64_t C)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < C) geom[c].cell_base = base[c];
}

__global__ void k_bin(panna_system sys, int S, const CfgGeom* __restrict__ geom,
                      const int32_t* __restrict__ atom_cfg, int32_t* __restrict__ atom_cell,
                      int64_t* __restrict__ cell_count, float4* __restrict__ pos_hi,
                      float4* __restrict__ pos_lo, int32_t* __restrict__ wrap, DevStatus* st)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= sys.n_atoms) return;
    const int c = atom_cfg[i];
    const CfgGeom& g = geom[c];
    double x[3] = {sys.pos[3 * i], sys.pos[3 * i + 1], sys.pos[3 * i + 2]};
    int sp = sys.species[i];
    if (sp < 0 || sp >= S) { set_status(st, PANNA_ERR_BAD_INPUT, (int)i); sp = 0; }
    if (!(isfinite(x[0]) && isfinite(x[1]) && isfinite(x[2]))) {
        set_status(st, PANNA_ERR_BAD_INPUT, (int)i);
        x[0] = x[1] = x[2] = 0.0;
    }
    int m[3], ci[3];
    double sf[3];
    for (int a = 0; a < 3; ++a) {
        double s = x[0] * g.cinv[a] + x[1] * g.cinv[3 + a] + x[2] * g.cinv[6 + a];
        m[a] = g.per[a] ? -(int)floor(s) : 0;
        sf[a] = s + m[a];
        double q = floor((sf[a] - g.lo[a]) * g.inv_w[a]);
        int k = q < 0.0 ? 0 : (q >= (double)g.n[a] ? g.n[a] - 1 : (int)q);
        ci[a] = k;
    }
    double xw[3];
    for (int d = 0; d < 3; ++d) xw[d] = x[d] + m[0] * g.cell[d] + m[1] * g.cell[3 + d] + m[2] * g.cell[6 + d];
    float h0 = (float)xw[0], h1 = (float)xw[1], h2 = (float)xw[2];
    pos_hi[i] = make_float4(h0, h1, h2, __int_as_float(sp));
    pos_lo[i] = make_float4((float)(xw[0] - h0), (float)(xw[1] - h1), (float)(xw[2] - h2), 0.f);
    wrap[3 * i] = m[0]; wrap[3 * i + 1] = m[1]; wrap[3 * i + 2] = m[2];
    int local = (ci[0] * g.n[1] + ci[1]) * g.n[2] + ci[2];
    atom_cell[i] = local;
    atomicAdd((unsigned long long*)&cell_count[g.cell_base + local], 1ull);
}

__global__ void k_scatter(int64_t N, const int32_t* __restrict__ atom_cfg, const int32_t* __restrict__ atom_cell,
                          const CfgGeom* __restrict__ geom, const int64_t* __restrict__ cell_start,
                          int32_t* __restrict__ cell_fill, int32_t* __restrict__ cell_atoms)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int64_t gc = geom[atom_cfg[i]].cell_base + atom_cell[i];
    int k = atomicAdd(&cell_fill[gc], 1);
    cell_atoms[cell_start[gc] + k] = (int32_t)i;
}

// atoms of each cell sorted by index; with pos_hi_s / pos_lo_s, the folded positions copied in
// that cell order (the candidate loop of the search then reads a candidate's position by its
// slot, not through its atom index).  Resident warps take the cells in use (the configurations'
// grids, read from the last configuration's geometry; the cell slots past them are empty) one
// cell per warp in turn.  A cell of up to 32 * kSortPer atoms is held in registers and each atom
// goes to slot b + (number of the cell's atoms with a smaller index), the indices being
// distinct; larger cells are sorted by insertion on one lane.
constexpr int kSortWarps = 8;
constexpr int kSortPer = 4;
constexpr int64_t kSortMaxWarps = 152 * 256;   // enough warps to fill every SM several times

__device__ __forceinline__ void sort_cell(int64_t b, int64_t e, int lane, int32_t* __restrict__ cell_atoms,
                                          const float4* __restrict__ pos_hi, const float4* __restrict__ pos_lo,
                                          float4* __restrict__ pos_hi_s, float4* __restrict__ pos_lo_s)
{
    const int64_t n = e - b;
    if (n <= 32 * kSortPer) {
        int32_t v[kSortPer];
        int rank[kSortPer];
#pragma unroll
        for (int t = 0; t < kSortPer; ++t) {
            const int64_t k = lane + 32 * t;
            v[t] = k < n ? cell_atoms[b + k] : INT32_MAX;
            rank[t] = 0;
        }
#pragma unroll
        for (int u = 0; u < kSortPer; ++u) {
            const int64_t left = n - 32 * u;
            const int m = left < 32 ? (int)left : 32;   // atoms held in the lanes' v[u]
            if (m <= 0) break;
            for (int src = 0; src < m; ++src) {
                const int32_t y = __shfl_sync(0xffffffffu, v[u], src);
#pragma unroll
                for (int t = 0; t < kSortPer; ++t) rank[t] += y < v[t] ? 1 : 0;
            }
        }
        __syncwarp();   // every lane has read its atoms before any slot is rewritten
#pragma unroll
        for (int t = 0; t < kSortPer; ++t) {
            if (lane + 32 * t >= n) continue;
            const int64_t k = b + rank[t];
            cell_atoms[k] = v[t];
            if (pos_hi_s) {
                pos_hi_s[k] = pos_hi[v[t]];
                pos_lo_s[k] = pos_lo[v[t]];
            }
        }
        __syncwarp();
        return;
    }
    if (lane == 0) {
        for (int64_t k = b + 1; k < e; ++k) {
            int32_t v = cell_atoms[k];
            int64_t q = k - 1;
            while (q >= b && cell_atoms[q] > v) { cell_atoms[q + 1] = cell_atoms[q]; --q; }
            cell_atoms[q + 1] = v;
        }
    }
    __syncwarp();   // lane 0's writes are visible to the warp after this
    if (pos_hi_s) {
        for (int64_t k = b + lane; k < e; k += 32) {
            const int32_t j = cell_atoms[k];
            pos_hi_s[k] = pos_hi[j];
            pos_lo_s[k] = pos_lo[j];
        }
    }
    __syncwarp();
}

__global__ void __launch_bounds__(kSortWarps * 32)
k_sort_cells(int64_t C, const CfgGeom* __restrict__ geom, int64_t ncells, const int64_t* __restrict__ cell_start,
             int32_t* __restrict__ cell_atoms, const float4* __restrict__ pos_hi, const float4* __restrict__ pos_lo,
             float4* __restrict__ pos_hi_s, float4* __restrict__ pos_lo_s)
{
    const int lane = threadIdx.x & 31;
    int64_t used = geom[C - 1].cell_base + geom[C - 1].ncells;
    if (used > ncells) used = ncells;
    const int64_t stride = (int64_t)gridDim.x * kSortWarps;
    for (int64_t c = (int64_t)blockIdx.x * kSortWarps + (threadIdx.x >> 5); c < used; c += stride) {
        const int64_t b = cell_start[c], e = cell_start[c + 1];
        if (e > b) sort_cell(b, e, lane, cell_atoms, pos_hi, pos_lo, pos_hi_s, pos_lo_s);
    }
}

// ------------------------------------------------------------------ neighbour search

// error-free sum of two floats: s + err == a + b exactly
__device__ __forceinline__ float two_sum(float a, float b, float& err)
{
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}

// (xj + S) - xi with each operand given as hi + lo, to about one FP32 rounding; lo receives
// what the rounded result leaves of the double-float value (about 2^-46 of it)
__device__ __forceinline__ float dd_rel(float xjh, float xjl, float sh, float sl, float xih, float xil, float& lo)
{
    float e1, e2;
    float a = two_sum(xjh, sh, e1);
    float b = two_sum(a, -xih, e2);
    float tail = __fsub_rn(__fadd_rn(__fadd_rn(e1, e2), __fadd_rn(xjl, sl)), xil);
    return two_sum(b, tail, lo);
}

constexpr int kNbWarps = 8;
constexpr int kNbQueue = 64;   // candidates within the filter band awaiting the exact test

// per-warp tables of the candidate loop: the current batch of 32 window cells (candidate
// offsets, first slot, image shift hi with the packed image code, shift lo) and the queue of
// filtered candidates (slot in cell order, cell of the batch)
struct NbWarpTables {
    int pre[33];
    int beg[32];
    float4 shA[32];
    float4 shB[32];
    int4 queue[kNbQueue];
};

// Rare paths with FP64 arithmetic, kept out of line: GB300 runs FP64 at 1/64 of the FP32
// rate, and the hot loop must not carry (even predicated-off) FP64 instructions.
struct Shift6 {
    float h0, h1, h2, l0, l1, l2;   // image shift as hi + lo floats
};

__device__ __noinline__ Shift6 shift_hilo(const CfgGeom& g, int t0, int t1, int t2)
{
    Shift6 r;
    float h[3], l[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double Sv = t0 * g.cell[d] + t1 * g.cell[3 + d] + t2 * g.cell[6 + d];
        h[d] = (float)Sv;
        l[d] = (float)(Sv - (double)h[d]);
    }
    r.h0 = h[0]; r.h1 = h[1]; r.h2 = h[2]; r.l0 = l[0]; r.l1 = l[1]; r.l2 = l[2];
    return r;
}

__device__ __noinline__ bool retest_fp64(float4 xjh, float4 xjl, Shift6 sh, float4 xih, float4 xil, double rc2d)
{
    double rx = ((double)xjh.x + (double)xjl.x) + ((double)sh.h0 + (double)sh.l0) - ((double)xih.x + (double)xil.x);
    double ry = ((double)xjh.y + (double)xjl.y) + ((double)sh.h1 + (double)sh.l1) - ((double)xih.y + (double)xil.y);
    double rz = ((double)xjh.z + (double)xjl.z) + ((double)sh.h2 + (double)sh.l2) - ((double)xih.z + (double)xil.z);
    return (rx * rx + ry * ry + rz * rz) < rc2d;
}

// 4 CTAs of 8 warps per SM (64 registers): the search waits on its candidate loads
__global__ void __launch_bounds__(kNbWarps * 32, 4)
k_neighbors(int64_t N, int S, double rc_d, float rc, const CfgGeom* __restrict__ geom,
            const int32_t* __restrict__ atom_cfg, const int32_t* __restrict__ atom_cell,
            const int64_t* __restrict__ cell_start, const int32_t* __restrict__ cell_atoms,
            const float4* __restrict__ pos_hi, const float4* __restrict__ pos_lo,
            const float4* __restrict__ pos_hi_s, const float4* __restrict__ pos_lo_s, int cap,
            const uint8_t* __restrict__ ghost, int32_t* __restrict__ nb_count, float4* __restrict__ nb_vec,
            int2* __restrict__ nb_idx, float4* __restrict__ nb_vlo, DevStatus* st)
{
    extern __shared__ unsigned char smem_raw[];
    __shared__ NbWarpTables nb_tables[kNbWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4* svec = reinterpret_cast<float4*>(smem_raw) + (size_t)warp * cap;
    int2* sidx = reinterpret_cast<int2*>(reinterpret_cast<float4*>(smem_raw) + (size_t)kNbWarps * cap) + (size_t)warp * cap;
    // low parts of the vectors (only with nb_vlo), after the index slots
    float4* svlo = reinterpret_cast<float4*>(reinterpret_cast<int2*>(reinterpret_cast<float4*>(smem_raw) +
                                                                     (size_t)kNbWarps * cap) + (size_t)kNbWarps * cap) +
                   (size_t)warp * cap;
    // warps take the atoms in cell order (cell_atoms is a permutation of the atoms): the warps
    // of a CTA scan overlapping windows of cells, so candidate positions come from L1
    const int64_t gw = (int64_t)blockIdx.x * kNbWarps + warp;
    if (gw >= N) return;
    const int64_t i = cell_atoms[gw];
    if (i < 0 || i >= N) return;   // not reached: every atom is binned into exactly one cell
    if (ghost && ghost[i]) {          // a ghost is a neighbour only, never a centre
        if (lane == 0) nb_count[i] = 0;
        return;
    }
    const int c = atom_cfg[i];
    const CfgGeom& g = geom[c];
    const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
    const int local = atom_cell[i];
    const int ci0 = local / (n1 * n2), ci1 = (local / n2) % n1, ci2 = local % n2;
    const float4 xih = pos_hi[i], xil = pos_lo[i];
    const float band = rc + 1e-2f;
    const float band2 = band * band;
    const float rc2 = rc * rc;
    const double rc2d = rc_d * rc_d;
    const unsigned lt = (1u << lane) - 1u;
    int count = 0;
    // The window of (2K+1)^3 cells around the atom's cell, 32 cells at a time (one per lane):
    // each lane resolves its cell (periodic wrap, image shift, atom range) into the warp's cell
    // table, a warp scan gives every cell's offset in the concatenated candidate list, and the
    // lanes take the candidates 32 at a time, each finding its cell by a binary search over the
    // offsets.  The filter on the FP32 hi parts (within rc + 0.01 A) is all a candidate costs;
    // those that pass go to a per-warp queue, and only the queue's entries, 32 at a time, get
    // the double-float relative vector, the cutoff test and the output.  Cells are visited in
    // the order of a nested (d0, d1, d2) loop, atoms in cell order, and the queue keeps that
    // order, so the neighbour order is deterministic.
    NbWarpTables& tb = nb_tables[warp];
    const int W1 = 2 * g.K[1] + 1, W2 = 2 * g.K[2] + 1;
    const int nwin = (2 * g.K[0] + 1) * W1 * W2;
    int qhead = 0, qtail = 0;
    // dense round over queue entries qhead .. qhead + m - 1
    auto process = [&](int m) {
        bool in = false;
        float dx = 0.f, dy = 0.f, dz = 0.f, r2 = 0.f, lx = 0.f, ly = 0.f, lz = 0.f;
        int j = -1, tc = 0, spj = 0;
        if (lane < m) {
            const int4 e = tb.queue[(qhead + lane) & (kNbQueue - 1)];
            j = cell_atoms[e.x];
            const float4 xjh = pos_hi_s[e.x], xjl = pos_lo_s[e.x];
            const float4 ta = tb.shA[e.y], tbl = tb.shB[e.y];
            tc = __float_as_int(ta.w);
            spj = __float_as_int(xjh.w);
            dx = dd_rel(xjh.x, xjl.x, ta.x, tbl.x, xih.x, xil.x, lx);
            dy = dd_rel(xjh.y, xjl.y, ta.y, tbl.y, xih.y, xil.y, ly);
            dz = dd_rel(xjh.z, xjl.z, ta.z, tbl.z, xih.z, xil.z, lz);
            r2 = __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz)));
            if (fabsf(r2 - rc2) <= 2e-6f * rc2) {
                const Shift6 cs{ta.x, ta.y, ta.z, tbl.x, tbl.y, tbl.z};
                in = retest_fp64(xjh, xjl, cs, xih, xil, rc2d);   // FP64 near the cutoff
            } else {
                in = r2 < rc2;
            }
            if (in && r2 == 0.f) { set_status(st, PANNA_ERR_BAD_INPUT, (int)i); in = false; }
        }
        const unsigned mask = __ballot_sync(0xffffffffu, in);
        if (in) {
            const int pos = count + __popc(mask & lt);
            if (pos < cap) {
                svec[pos] = make_float4(dx, dy, dz, sqrtf(r2));
                sidx[pos] = make_int2(j, tc | (spj << 24));
                if (nb_vlo) svlo[pos] = make_float4(lx, ly, lz, 0.f);
            }
        }
        count += __popc(mask);
        qhead += m;
    };
    for (int cb = 0; cb < nwin; cb += 32) {
        const int wc = cb + lane;
        int cnt = 0, tcode = 0;
        int64_t beg = 0;
        Shift6 sh{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (wc < nwin) {
            const int d0 = wc / (W1 * W2) - g.K[0], d1 = (wc / W2) % W1 - g.K[1], d2 = wc % W2 - g.K[2];
            int c0 = ci0 + d0, c1 = ci1 + d1, c2 = ci2 + d2, t0 = 0, t1 = 0, t2 = 0;
            bool ok = true;
            if (g.per[0]) { t0 = (c0 >= 0 ? c0 / n0 : -((-c0 + n0 - 1) / n0)); c0 -= t0 * n0; }
            else ok = ok && c0 >= 0 && c0 < n0;
            if (g.per[1]) { t1 = (c1 >= 0 ? c1 / n1 : -((-c1 + n1 - 1) / n1)); c1 -= t1 * n1; }
            else ok = ok && c1 >= 0 && c1 < n1;
            if (g.per[2]) { t2 = (c2 >= 0 ? c2 / n2 : -((-c2 + n2 - 1) / n2)); c2 -= t2 * n2; }
            else ok = ok && c2 >= 0 && c2 < n2;
            if (ok) {
                const int64_t gc = g.cell_base + (c0 * n1 + c1) * n2 + c2;
                beg = cell_start[gc];
                cnt = (int)(cell_start[gc + 1] - beg);
                tcode = pack_meta(t0, t1, t2, 0);
                if (t0 >= -1 && t0 <= 1 && t1 >= -1 && t1 <= 1 && t2 >= -1 && t2 <= 1) {
                    const int k = (t0 + 1) * 9 + (t1 + 1) * 3 + (t2 + 1);
                    sh = Shift6{g.sh_hi[k][0], g.sh_hi[k][1], g.sh_hi[k][2], g.sh_lo[k][0], g.sh_lo[k][1],
                                g.sh_lo[k][2]};
                } else {
                    sh = shift_hilo(g, t0, t1, t2);
                }
            }
        }
        // exclusive offsets of the cells' candidates
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        tb.pre[lane] = incl - cnt;
        tb.beg[lane] = (int)beg;
        tb.shA[lane] = make_float4(sh.h0, sh.h1, sh.h2, __int_as_float(tcode));
        tb.shB[lane] = make_float4(sh.l0, sh.l1, sh.l2, 0.f);
        __syncwarp();
        for (int base = 0; base < total; base += 32) {
            const int q = base + lane;
            bool band = false;
            int slot = 0, sl = 0;
            if (q < total) {
                // the cell of candidate q: the last cell whose offset is <= q (empty cells share
                // an offset with the next one and lose the search)
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1)
                    if (tb.pre[sl + step] <= q) sl += step;
                slot = tb.beg[sl] + (q - tb.pre[sl]);
                const float4 xjh = pos_hi_s[slot];
                const float4 ta = tb.shA[sl];
                const float fx = (xjh.x + ta.x) - xih.x;
                const float fy = (xjh.y + ta.y) - xih.y;
                const float fz = (xjh.z + ta.z) - xih.z;
                const float f2 = fx * fx + fy * fy + fz * fz;
                // the atom itself (unshifted image, its own slot in cell order) is no neighbour
                const bool self = (__float_as_int(ta.w) & 0xffffff) == pack_meta(0, 0, 0, 0) && slot == (int)gw;
                band = f2 < band2 && !self;
            }
            const unsigned bm = __ballot_sync(0xffffffffu, band);
            if (band) tb.queue[(qtail + __popc(bm & lt)) & (kNbQueue - 1)] = make_int4(slot, sl, 0, 0);
            qtail += __popc(bm);
            __syncwarp();
            if (qtail - qhead >= 32) {
                process(32);
                __syncwarp();
            }
        }
        // the next batch of cells rewrites the table: finish the queue first
        if (qtail > qhead) process(qtail - qhead);
        __syncwarp();
    }
    if (count > cap && lane == 0) {
        atomicMax(&st->need_cap, count);
        set_status(st, PANNA_ERR_NEIGHBOR_OVERFLOW, (int)i);
    }
    const int n = count < cap ? count : cap;
    if (lane == 0) nb_count[i] = n;
    __syncwarp();
    const size_t out = (size_t)i * cap;
    if (S == 1) {
        for (int k = lane; k < n; k += 32) {
            nb_vec[out + k] = svec[k];
            nb_idx[out + k] = sidx[k];
            if (nb_vlo) nb_vlo[out + k] = svlo[k];
        }
        return;
    }
    int w = 0;
    for (int s = 0; s < S; ++s) {
        for (int base = 0; base < n; base += 32) {
            const int k = base + lane;
            const bool take = k < n && meta_species(sidx[k].y) == s;
            const unsigned mask = __ballot_sync(0xffffffffu, take);
            if (take) {
                const int p = w + __popc(mask & lt);
                nb_vec[out + p] = svec[k];
                nb_idx[out + p] = sidx[k];
                if (nb_vlo) nb_vlo[out + p] = svlo[k];
            }
            w += __popc(mask);
        }
    }
}

// ------------------------------------------------------------------ Verlet-list refresh

// Positions folded with the lattice offsets recorded when the list was built (wrap), so the
// image shifts stored with the candidates stay valid while atoms move; species in .w kept.
__global__ void k_fold_frozen(int64_t N, const double* __restrict__ pos, const int32_t* __restrict__ atom_cfg,
                              const CfgGeom* __restrict__ geom, const int32_t* __restrict__ wrap,
                              float4* __restrict__ pos_hi, float4* __restrict__ pos_lo)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const CfgGeom& g = geom[atom_cfg[i]];
    const int m0 = wrap[3 * i], m1 = wrap[3 * i + 1], m2 = wrap[3 * i + 2];
    double xw[3];
    for (int d = 0; d < 3; ++d) xw[d] = pos[3 * i + d] + m0 * g.cell[d] + m1 * g.cell[3 + d] + m2 * g.cell[6 + d];
    const float h0 = (float)xw[0], h1 = (float)xw[1], h2 = (float)xw[2];
    const float w = pos_hi[i].w;
    pos_hi[i] = make_float4(h0, h1, h2, w);
    pos_lo[i] = make_float4((float)(xw[0] - h0), (float)(xw[1] - h1), (float)(xw[2] - h2), 0.f);
}

// The candidates (j, image) found within rc + skin when the list was built are re-tested
// at the current positions with the arithmetic of the full search (FP32 band filter,
// double-float relative vector, FP64 re-test near rc); those with r < rc are kept in their
// stored order (grouped by species).  Exact as long as no atom has moved more than skin/2
// since the build (every pair now within rc was then within rc + skin).
__global__ void __launch_bounds__(kNbWarps * 32)
k_refresh(int64_t N, double rc_d, float rc, const CfgGeom* __restrict__ geom, const int32_t* __restrict__ atom_cfg,
          const int32_t* __restrict__ cand_count, const int2* __restrict__ cand_idx, int cap_c,
          const float4* __restrict__ pos_hi, const float4* __restrict__ pos_lo, int cap,
          int32_t* __restrict__ nb_count, float4* __restrict__ nb_vec, int2* __restrict__ nb_idx,
          float4* __restrict__ nb_vlo, DevStatus* st)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * kNbWarps + warp;
    if (i >= N) return;
    const CfgGeom& g = geom[atom_cfg[i]];
    const float4 xih = pos_hi[i], xil = pos_lo[i];
    const float band = rc + 1e-2f, band2 = band * band, rc2 = rc * rc;
    const double rc2d = rc_d * rc_d;
    const unsigned lt = (1u << lane) - 1u;
    const int nc = min(cand_count[i], cap_c);
    const size_t cin = (size_t)i * cap_c, out = (size_t)i * cap;
    int count = 0;
    for (int base = 0; base < nc; base += 32) {
        const int k = base + lane;
        bool in = false;
        float dx = 0.f, dy = 0.f, dz = 0.f, r2 = 0.f, lx = 0.f, ly = 0.f, lz = 0.f;
        int2 e = make_int2(0, 0);
        if (k < nc) {
            e = cand_idx[cin + k];
            const int t0 = meta_t(e.y, 0), t1 = meta_t(e.y, 1), t2 = meta_t(e.y, 2);
            Shift6 cs;
            if (t0 >= -1 && t0 <= 1 && t1 >= -1 && t1 <= 1 && t2 >= -1 && t2 <= 1) {
                const int q = (t0 + 1) * 9 + (t1 + 1) * 3 + (t2 + 1);
                cs = Shift6{g.sh_hi[q][0], g.sh_hi[q][1], g.sh_hi[q][2], g.sh_lo[q][0], g.sh_lo[q][1], g.sh_lo[q][2]};
            } else {
                cs = shift_hilo(g, t0, t1, t2);
            }
            const float4 xjh = pos_hi[e.x];
            const float fx = (xjh.x + cs.h0) - xih.x, fy = (xjh.y + cs.h1) - xih.y, fz = (xjh.z + cs.h2) - xih.z;
            if (fx * fx + fy * fy + fz * fz < band2) {
                const float4 xjl = pos_lo[e.x];
                dx = dd_rel(xjh.x, xjl.x, cs.h0, cs.l0, xih.x, xil.x, lx);
                dy = dd_rel(xjh.y, xjl.y, cs.h1, cs.l1, xih.y, xil.y, ly);
                dz = dd_rel(xjh.z, xjl.z, cs.h2, cs.l2, xih.z, xil.z, lz);
                r2 = __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz)));
                if (fabsf(r2 - rc2) <= 2e-6f * rc2) in = retest_fp64(xjh, xjl, cs, xih, xil, rc2d);
                else in = r2 < rc2;
                if (in && r2 == 0.f) { set_status(st, PANNA_ERR_BAD_INPUT, (int)i); in = false; }
            }
        }
        const unsigned mask = __ballot_sync(0xffffffffu, in);
        if (in) {
            const int p = count + __popc(mask & lt);
            if (p < cap) {
                nb_vec[out + p] = make_float4(dx, dy, dz, sqrtf(r2));
                nb_idx[out + p] = e;
                if (nb_vlo) nb_vlo[out + p] = make_float4(lx, ly, lz, 0.f);
            }
        }
        count += __popc(mask);
    }
    if (count > cap && lane == 0) {
        atomicMax(&st->need_cap, count);
        set_status(st, PANNA_ERR_NEIGHBOR_OVERFLOW, (int)i);
    }
    if (lane == 0) nb_count[i] = count < cap ? count : cap;
}

cudaError_t refresh_neighbors(const Work& cand, Work& w, const DescDev& d, cudaStream_t s, int* launches)
{
    const int64_t N = w.N;
    if (N == 0) return cudaSuccess;
    k_fold_frozen<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, w.sys->pos, w.atom_cfg, w.geom, w.wrap, w.pos_hi,
                                                              w.pos_lo);
    k_refresh<<<(unsigned)((N + kNbWarps - 1) / kNbWarps), kNbWarps * 32, 0, s>>>(
        N, d.rc_d, d.rc, w.geom, w.atom_cfg, cand.nb_count, cand.nb_idx, cand.cap, w.pos_hi, w.pos_lo, w.cap,
        w.nb_count, w.nb_vec, w.nb_idx, w.nb_vlo, w.status);
    *launches += 2;
    return cudaGetLastError();
}

// ------------------------------------------------------------------ CSR export

__global__ void k_count_i64(int64_t N, const int32_t* __restrict__ cnt, int64_t* __restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) out[i] = cnt[i];
}

__global__ void k_export(int64_t N, int cap, const int32_t* __restrict__ nb_count, const int2* __restrict__ nb_idx,
                         const int32_t* __restrict__ wrap, const int64_t* __restrict__ off, int64_t cap_total,
                         int64_t* __restrict__ nbr_j, int32_t* __restrict__ shift)
{
    int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= N) return;
    const int n = nb_count[i];
    for (int k = lane; k < n; k += 32) {
        const int64_t p = off[i] + k;
        if (p >= cap_total) continue;
        const int2 e = nb_idx[(size_t)i * cap + k];
        nbr_j[p] = e.x;
        for (int a = 0; a < 3; ++a) shift[3 * p + a] = wrap[3 * (int64_t)e.x + a] - wrap[3 * i + a] + meta_t(e.y, a);
    }
}

cudaError_t export_neighbors(const Work& w, int64_t* off, int64_t* nbr_j, int32_t* shift, int64_t cap_total,
                             cudaStream_t s, int* launches)
{
    const int64_t N = w.N;
    unsigned nb = (unsigned)((N + 255) / 256);
    if (nb == 0) nb = 1;
    k_count_i64<<<nb, 256, 0, s>>>(N, w.nb_count, w.cell_count);
    ++*launches;
    cudaError_t e = exclusive_scan_i64(w.cell_count, off, N, w.scan_tmp, s, launches);
    if (e != cudaSuccess) return e;
    unsigned nw = (unsigned)((N + 7) / 8);
    if (nw == 0) nw = 1;
    k_export<<<nw, 256, 0, s>>>(N, w.cap, w.nb_count, w.nb_idx, w.wrap, off, cap_total, nbr_j, shift);
    ++*launches;
    return cudaGetLastError();
}

// ------------------------------------------------------------------ driver

cudaError_t build_neighbors(Work& w, const DescDev& d, cudaStream_t s, int* launches)
{
    const int64_t N = w.N, C = w.C;
    const panna_system& sys = *w.sys;
    cudaError_t e;
    unsigned nbA = (unsigned)((N + 255) / 256);
    if (nbA == 0) nbA = 1;
    k_atom_cfg<<<nbA, 256, 0, s>>>(sys.atom_off, C, N, w.atom_cfg);
    k_cfg_geom<<<(unsigned)((C + kCfgWarps - 1) / kCfgWarps), kCfgWarps * 32, 0, s>>>(sys, d.rc_d, w.geom,
                                                                                      w.cell_count, w.status);
    *launches += 2;
    // cell bases: scan of per-config cell counts (stored temporarily in cell_count[0..C))
    e = exclusive_scan_i64(w.cell_count, w.cell_start, C, w.scan_tmp, s, launches);
    if (e != cudaSuccess) return e;
    k_set_cell_base<<<(unsigned)((C + 255) / 256), 256, 0, s>>>(w.geom, w.cell_start, C);
    ++*launches;
    // total cells <= 2N + C by construction; clear the counters
    e = cudaMemsetAsync(w.cell_count, 0, sizeof(int64_t) * (w.cap_cells + 1), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(w.cell_fill, 0, sizeof(int32_t) * w.cap_cells, s);
    if (e != cudaSuccess) return e;
    k_bin<<<nbA, 256, 0, s>>>(sys, d.S, w.geom, w.atom_cfg, w.atom_cell, w.cell_count, w.pos_hi, w.pos_lo,
                              w.wrap, w.status);
    ++*launches;
    e = exclusive_scan_i64(w.cell_count, w.cell_start, w.cap_cells, w.scan_tmp, s, launches);
    if (e != cudaSuccess) return e;
    k_scatter<<<nbA, 256, 0, s>>>(N, w.atom_cfg, w.atom_cell, w.geom, w.cell_start, w.cell_fill, w.cell_atoms);
    {
        const int64_t warps = std::min<int64_t>(w.cap_cells, kSortMaxWarps);
        k_sort_cells<<<(unsigned)((warps + kSortWarps - 1) / kSortWarps), kSortWarps * 32, 0, s>>>(
            C, w.geom, w.cap_cells, w.cell_start, w.cell_atoms, w.pos_hi, w.pos_lo, w.pos_hi_s, w.pos_lo_s);
    }
    *launches += 2;
    size_t smem = (size_t)kNbWarps * w.cap * (sizeof(float4) + sizeof(int2) + (w.nb_vlo ? sizeof(float4) : 0));
    e = cudaFuncSetAttribute(k_neighbors, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    unsigned nbW = (unsigned)((N + kNbWarps - 1) / kNbWarps);
    if (nbW == 0) nbW = 1;
    k_neighbors<<<nbW, kNbWarps * 32, smem, s>>>(N, d.S, d.rc_d, d.rc, w.geom, w.atom_cfg, w.atom_cell,
                                                 w.cell_start, w.cell_atoms, w.pos_hi, w.pos_lo, w.pos_hi_s,
                                                 w.pos_lo_s, w.cap,
                                                 w.sys->ghost, w.nb_count, w.nb_vec, w.nb_idx, w.nb_vlo, w.status);
    ++*launches;
    return cudaGetLastError();
}

// ------------------------------------------------------------------ species order

constexpr int kSpBlock = 1024;

// Rows of the networks: the non-ghost atoms grouped by species (ghosts get row -1).
__global__ void k_species_count(int64_t N, int S, const float4* __restrict__ pos_hi, const uint8_t* __restrict__ ghost,
                                int32_t* __restrict__ blk_counts)
{
    __shared__ int cnt[kMaxSpecies];
    if (threadIdx.x < kMaxSpecies) cnt[threadIdx.x] = 0;
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * kSpBlock + threadIdx.x;
    if (i < N && !(ghost && ghost[i])) atomicAdd(&cnt[__float_as_int(pos_hi[i].w)], 1);
    __syncthreads();
    if (threadIdx.x < S) blk_counts[(size_t)blockIdx.x * S + threadIdx.x] = cnt[threadIdx.x];
}

constexpr int kOffThreads = 1024;

// Offsets of every (block, species) count: per species an exclusive scan over the blocks (one
// CTA; each thread walks a contiguous run of blocks, a block-wide scan joins the runs), shifted
// by the totals of the species before it; seg_off[s] = first row of species s.
__global__ void __launch_bounds__(kOffThreads)
k_species_offsets(int64_t nblk, int S, int32_t* __restrict__ blk_counts, int32_t* __restrict__ seg_off)
{
    __shared__ int wsum[kOffThreads / 32];
    __shared__ int s_base;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int64_t per = (nblk + kOffThreads - 1) / kOffThreads;
    const int64_t b0 = min(nblk, (int64_t)t * per), b1 = min(nblk, b0 + per);
    if (t == 0) s_base = 0;
    __syncthreads();
    for (int s = 0; s < S; ++s) {
        int sum = 0;
        for (int64_t b = b0; b < b1; ++b) sum += blk_counts[b * S + s];
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) wsum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int v = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += u;
            }
            wsum[lane] = v;
        }
        __syncthreads();
        const int base = s_base;
        int run = base + (wid > 0 ? wsum[wid - 1] : 0) + incl - sum;
        for (int64_t b = b0; b < b1; ++b) {
            const int v = blk_counts[b * S + s];
            blk_counts[b * S + s] = run;
            run += v;
        }
        __syncthreads();   // base and the warp sums are read
        if (t == 0) {
            seg_off[s] = base;
            s_base = base + wsum[kOffThreads / 32 - 1];
        }
        __syncthreads();
    }
    if (t == 0) seg_off[S] = s_base;
}

__global__ void k_species_rank(int64_t N, int S, const float4* __restrict__ pos_hi, const uint8_t* __restrict__ ghost,
                               const int32_t* __restrict__ blk_off, int32_t* __restrict__ row_of_atom,
                               int32_t* __restrict__ atom_of_row)
{
    __shared__ int wcnt[kSpBlock / 32][kMaxSpecies];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t i = (int64_t)blockIdx.x * kSpBlock + threadIdx.x;
    int sp = (i < N && !(ghost && ghost[i])) ? __float_as_int(pos_hi[i].w) : -1;
    int my_rank = 0;
    for (int s = 0; s < S; ++s) {
        unsigned m = __ballot_sync(0xffffffffu, sp == s);
        if (sp == s) my_rank = __popc(m & ((1u << lane) - 1u));
        if (lane == 0) wcnt[wid][s] = __popc(m);
    }
    __syncthreads();
    if (i < N && sp < 0) row_of_atom[i] = -1;
    if (i < N && sp >= 0) {
        int before = 0;
        for (int w2 = 0; w2 < wid; ++w2) before += wcnt[w2][sp];
        int row = blk_off[(size_t)blockIdx.x * S + sp] + before + my_rank;
        row_of_atom[i] = row;
        atom_of_row[row] = (int32_t)i;
    }
}

cudaError_t species_order(Work& w, int S, cudaStream_t s, int* launches)
{
    int64_t nblk = (w.N + kSpBlock - 1) / kSpBlock;
    if (nblk == 0) nblk = 1;
    const uint8_t* ghost = w.sys->ghost;
    k_species_count<<<(unsigned)nblk, kSpBlock, 0, s>>>(w.N, S, w.pos_hi, ghost, w.blk_counts);
    k_species_offsets<<<1, kOffThreads, 0, s>>>(nblk, S, w.blk_counts, w.seg_off);
    k_species_rank<<<(unsigned)nblk, kSpBlock, 0, s>>>(w.N, S, w.pos_hi, ghost, w.blk_counts, w.row_of_atom,
                                                      w.atom_of_row);
    *launches += 3;
    return cudaGetLastError();
}

}  // namespace panna
