// Precomputed descriptors with stored Jacobians (Sec. II.A: the descriptors of a dataset
// are computed once and reused in every epoch, their derivatives stored beside them for
// the forces; the alternative is recomputing both in every step).
//
// A store holds, for one batch, the descriptor rows G in network order, the atom <-> row
// maps, the configuration of each atom, and per neighbour entry e = (i, j, n) its vector
// r_e and the non-zero part of J_e = dG_i/dr_e: the radial block of the neighbour's
// species and the S angular blocks that contain that species.  Columns per entry and
// Cartesian component: W = Rp + S Ap, with the radial width n_rad and the angular block
// width A = n_theta n_ang_r rounded up to multiples of 4 (Rp, Ap) so that a float4 never
// straddles two blocks; the padding columns hold zeros.
//
//   build (once):   J_e in FP64 from the positions, rounded to FP32;
//   forces:         q_e = g_i . J_e (g_i = dE_i/dG_i); F_i += sum_e q_e, F_j(e) -= q_e;
//                   per-atom virial -sum_e q_e (x) r_e;
//   tangent:        w_i = sum_e J_e (u_j(e) - u_i)  (the descriptor JVP of the weight
//                   gradient's force term).
// The two per-step kernels stream J once each: they are bound by HBM bandwidth, where the
// on-the-fly kernels recompute the angular terms and are bound by arithmetic.
#include <math.h>

#include "common.cuh"

namespace panna {

namespace {

__host__ __device__ inline int pair_block_s(int a, int b, int S)
{
    return a * S - a * (a - 1) / 2 + (b - a);
}

}  // namespace

void store_dims(const DescDev& d, StoreView& v)
{
    const int A = d.n_theta * d.n_ang_r;
    v.S = d.S;
    v.D = d.D;
    v.Rp = (d.n_rad + 3) & ~3;
    v.Ap = (A + 3) & ~3;
    v.W = v.Rp + d.S * v.Ap;
}

int64_t store_carve(StoreView& v, char* base, int64_t* off)
{
    int64_t pos = 0;
    int k = 0;
    auto take = [&](int64_t bytes) -> char* {
        pos = (pos + 255) & ~(int64_t)255;
        if (off) off[k] = pos;
        ++k;
        char* p = base ? base + pos : nullptr;
        pos += bytes;
        return p;
    };
    const int64_t N = v.N, P = v.P;
    v.G = reinterpret_cast<float*>(take(N * v.D * (int64_t)sizeof(float)));
    v.row_of_atom = reinterpret_cast<int32_t*>(take(N * 4));
    v.atom_of_row = reinterpret_cast<int32_t*>(take(N * 4));
    v.seg_off = reinterpret_cast<int32_t*>(take((v.S + 1) * 4));
    v.atom_cfg = reinterpret_cast<int32_t*>(take(N * 4));
    v.ent_off = reinterpret_cast<int64_t*>(take((N + 1) * 8));
    v.ent_idx = reinterpret_cast<int2*>(take(P * 8));
    v.ent_vec = reinterpret_cast<float4*>(take(P * 16));
    v.jac = reinterpret_cast<float*>(take(P * 3 * (int64_t)v.W * 4));
    return (pos + 255) & ~(int64_t)255;
}

// --------------------------------------------------------------------------- build

// FP64 vector of a neighbour slot m = (j, meta) of atom i: r = x_j - x_i + n.cell with the
// image n = wrap_j - wrap_i + t (t: shift between the folded positions)
__device__ __forceinline__ void entry_vector(const panna_system& sys, const Work& w, int64_t i, int2 m, int cfg,
                                             double r[3])
{
    const int64_t j = m.x;
    int nimg[3];
    for (int a = 0; a < 3; ++a) nimg[a] = w.wrap[3 * j + a] - w.wrap[3 * i + a] + meta_t(m.y, a);
    const double* cell = sys.cell + 9 * (int64_t)cfg;
    for (int a = 0; a < 3; ++a) {
        double x = sys.pos[3 * j + a] - sys.pos[3 * i + a];
        for (int b = 0; b < 3; ++b)
            if (nimg[b] != 0) x += nimg[b] * cell[3 * b + a];
        r[a] = x;
    }
}

__global__ void k_entry_counts(int64_t N, const int32_t* __restrict__ cnt, int64_t* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) out[i] = cnt[i];
}

cudaError_t launch_store_offsets(const Work& w, int64_t* off, cudaStream_t s, int* launches)
{
    const unsigned nb = (unsigned)((w.N + 255) / 256);
    if (nb > 0) {
        k_entry_counts<<<nb, 256, 0, s>>>(w.N, w.nb_count, w.cell_count);
        ++*launches;
    }
    return exclusive_scan_i64(w.cell_count, off, w.N, w.scan_tmp, s, launches);
}

constexpr int kEntWarps = 8;

__global__ void __launch_bounds__(kEntWarps * 32)
k_store_entries(panna_system sys, Work w, StoreView v)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * kEntWarps + warp;
    if (i >= w.N) return;
    const int n = w.nb_count[i];
    const int64_t e0 = v.ent_off[i];
    const int cfg = w.atom_cfg[i];
    for (int k = lane; k < n; k += 32) {
        const int2 m = w.nb_idx[(size_t)i * w.cap + k];
        double r[3];
        entry_vector(sys, w, i, m, cfg, r);
        v.ent_idx[e0 + k] = make_int2(m.x, meta_species(m.y));
        v.ent_vec[e0 + k] = make_float4((float)r[0], (float)r[1], (float)r[2],
                                        (float)sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]));
    }
}

cudaError_t launch_store_entries(const Work& w, const StoreView& v, cudaStream_t s, int* launches)
{
    const unsigned nb = (unsigned)((w.N + kEntWarps - 1) / kEntWarps);
    if (nb == 0) return cudaSuccess;
    k_store_entries<<<nb, kEntWarps * 32, 0, s>>>(*w.sys, w, v);
    ++*launches;
    return cudaGetLastError();
}

// x^n for n >= 0
__device__ __forceinline__ double ipow(double x, int n)
{
    double out = 1.0;
    while (n) {
        if (n & 1) out *= x;
        n >>= 1;
        if (n) x *= x;
    }
    return out;
}

// per-warp staging of the neighbour entries in FP64: |r|, unit vector, f_c, f_c'
constexpr int kJacStage = 6;

// One warp per centre atom.  Row k1 of the atom's entries: the radial columns of the
// neighbour's species, then for each species s the block {s_k1, s} summed over the partners
// k2 of species s (every unordered pair {k1, k2} contributes its derivative with respect to
// r_k1 to row k1 and with respect to r_k2 to row k2).  Lanes run over columns, so every
// value is one lane's sequential sum: the build is deterministic.
__global__ void k_store_jacobian(DescDev d, DescGrid64 g, panna_system sys, Work w, StoreView v)
{
    extern __shared__ double smd[];
    const int warps = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * warps + warp;
    if (i >= w.N) return;
    const int cap = w.cap;
    double* rr = smd + (size_t)warp * kJacStage * cap;
    double* ux = rr + cap; double* uy = ux + cap; double* uz = uy + cap;
    double* fc = uz + cap; double* dfc = fc + cap;
    const int n = w.nb_count[i];
    const int cfg = w.atom_cfg[i];
    for (int k = lane; k < n; k += 32) {
        const int2 m = w.nb_idx[(size_t)i * cap + k];
        double r[3];
        entry_vector(sys, w, i, m, cfg, r);
        const double len = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        rr[k] = len;
        ux[k] = r[0] / len; uy[k] = r[1] / len; uz[k] = r[2] / len;
        const double x = len / g.rc;
        fc[k] = len < g.rc ? 0.5 * (1.0 + cospi(x)) : 0.0;
        dfc[k] = len < g.rc ? -0.5 * (M_PI / g.rc) * sinpi(x) : 0.0;
    }
    // entries are grouped by species: segment starts
    int seg[kMaxSpecies + 1];
    {
        int cnt[kMaxSpecies];
#pragma unroll
        for (int s = 0; s < kMaxSpecies; ++s) cnt[s] = 0;
        for (int b0 = 0; b0 < n; b0 += 32) {
            const int k = b0 + lane;
            const int q = k < n ? meta_species(w.nb_idx[(size_t)i * cap + k].y) : -1;
#pragma unroll
            for (int s = 0; s < kMaxSpecies; ++s) cnt[s] += __popc(__ballot_sync(0xffffffffu, q == s));
        }
        seg[0] = 0;
#pragma unroll
        for (int s = 0; s < kMaxSpecies; ++s) seg[s + 1] = seg[s] + (s < d.S ? cnt[s] : 0);
    }
    __syncwarp();

    const int A = d.n_theta * d.n_ang_r, NA = d.n_ang_r;
    const int64_t e0 = v.ent_off[i];
    const int W = v.W;
    for (int k1 = 0; k1 < n; ++k1) {
        float* J = v.jac + (size_t)(e0 + k1) * 3 * W;
        const double r1 = rr[k1], f1 = fc[k1], df1 = dfc[k1];
        const double u1[3] = {ux[k1], uy[k1], uz[k1]};
        // radial block of the neighbour's species
        for (int c = lane; c < v.Rp; c += 32) {
            double dv = 0.0;
            if (c < d.n_rad) {
                const double x = r1 - g.rs_rad[c];
                const double ga = exp(-g.eta_rad * x * x);
                dv = ga * (-2.0 * g.eta_rad * x * f1 + df1);
            }
            J[c] = (float)(dv * u1[0]);
            J[W + c] = (float)(dv * u1[1]);
            J[2 * W + c] = (float)(dv * u1[2]);
        }
        // angular blocks {s_k1, s}
        for (int s = 0; s < d.S; ++s) {
            for (int c = lane; c < v.Ap; c += 32) {
                double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
                if (c < A) {
                    const int m = c / NA, q = c - m * NA;
                    const double ct = g.cos_t[m], st = g.sin_t[m], rs = g.rs_ang[q];
                    for (int k2 = seg[s]; k2 < seg[s + 1]; ++k2) {
                        if (k2 == k1) continue;
                        const double u2[3] = {ux[k2], uy[k2], uz[k2]};
                        const double cs = u1[0] * u2[0] + u1[1] * u2[1] + u1[2] * u2[2];
                        const double one_m = 1.0 - cs * cs;
                        const double sn = sqrt((one_m > 0.0 ? one_m : 0.0) + g.eps_theta);
                        const double dsn = one_m > 0.0 ? -cs / sn : 0.0;
                        const double bse = 1.0 + cs * ct + sn * st;
                        if (!(bse > 0.0)) continue;
                        const double p1 = g.zeta_int > 0 ? ipow(bse, g.zeta_int - 1) : pow(bse, g.zeta - 1.0);
                        const double Am = g.pref * p1 * bse;
                        const double dA = g.pref * g.zeta * p1 * (ct + dsn * st);
                        const double f2 = fc[k2];
                        const double x = 0.5 * (r1 + rr[k2]) - rs;
                        const double ga = exp(-g.eta_ang * x * x);
                        const double B = ga * f1 * f2;
                        const double dB1 = ga * (-g.eta_ang * x * f1 + df1) * f2;
                        // d cos / d r_k1 = (u2 - cos u1) / r1
                        const double a = dA * B / r1, b = Am * dB1;
                        acc0 += a * (u2[0] - cs * u1[0]) + b * u1[0];
                        acc1 += a * (u2[1] - cs * u1[1]) + b * u1[1];
                        acc2 += a * (u2[2] - cs * u1[2]) + b * u1[2];
                    }
                }
                const int col = v.Rp + s * v.Ap + c;
                J[col] = (float)acc0;
                J[W + col] = (float)acc1;
                J[2 * W + col] = (float)acc2;
            }
        }
    }
}

static int jac_warps(int cap)
{
    const size_t per = (size_t)kJacStage * cap * sizeof(double);
    int warps = (int)((200 * 1024) / per);
    return warps > 4 ? 4 : warps;
}

cudaError_t launch_store_jacobian(const Work& w, const DescDev& d, const DescGrid64& g, const StoreView& v,
                                  cudaStream_t s, int* launches)
{
    if (w.N == 0) return cudaSuccess;
    const int warps = jac_warps(w.cap);
    if (warps < 1) return cudaErrorInvalidValue;
    const size_t smem = (size_t)warps * kJacStage * w.cap * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_store_jacobian, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned nb = (unsigned)((w.N + warps - 1) / warps);
    k_store_jacobian<<<nb, warps * 32, smem, s>>>(d, g, *w.sys, w, v);
    ++*launches;
    return cudaGetLastError();
}

// --------------------------------------------------------------------------- per step

// Descriptor column of Jacobian column 4 c4 of an entry whose neighbour has species sj, and
// how many of the four consecutive columns are real (the rest is padding)
__device__ __forceinline__ void store_cols(const DescDev& d, const StoreView& v, int sj, int c4, int& gcol, int& valid)
{
    const int col = 4 * c4;
    if (col < v.Rp) {
        gcol = sj * d.n_rad + col;
        valid = d.n_rad - col;
    } else {
        const int ww = col - v.Rp;
        const int s = ww / v.Ap;
        const int loc = ww - s * v.Ap;
        const int A = d.n_theta * d.n_ang_r;
        gcol = d.rad_cols + pair_block_s(sj < s ? sj : s, sj < s ? s : sj, d.S) * A + loc;
        valid = A - loc;
    }
    valid = valid < 0 ? 0 : (valid > 4 ? 4 : valid);
}

constexpr int kStoreWarps = 8;

// q_e = g_i . J_e; forces and per-atom virial as the on-the-fly adjoint (one warp per atom)
template <bool VEC>
__global__ void __launch_bounds__(kStoreWarps * 32)
k_store_adjoint(StoreView v, DescDev d, const float* __restrict__ g_rows, float* __restrict__ F,
                float* __restrict__ vir_atom)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * kStoreWarps + warp;
    if (i >= v.N) return;
    const float* gi = g_rows + (size_t)v.row_of_atom[i] * d.D;
    const int64_t e0 = v.ent_off[i], e1 = v.ent_off[i + 1];
    const int W4 = v.W >> 2;
    float fx = 0.f, fy = 0.f, fz = 0.f;
    float vir[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) vir[k] = 0.f;
    for (int64_t e = e0; e < e1; ++e) {
        const int2 id = v.ent_idx[e];
        const float4* J0 = reinterpret_cast<const float4*>(v.jac + (size_t)e * 3 * v.W);
        const float4* J1 = J0 + W4;
        const float4* J2 = J1 + W4;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
        for (int c4 = lane; c4 < W4; c4 += 32) {
            const float4 x0 = __ldcs(J0 + c4), x1 = __ldcs(J1 + c4), x2 = __ldcs(J2 + c4);
            int gcol, valid;
            store_cols(d, v, id.y, c4, gcol, valid);
            float4 gv = make_float4(0.f, 0.f, 0.f, 0.f);
            if (VEC) {
                if (valid == 4) gv = *reinterpret_cast<const float4*>(gi + gcol);
            } else {
                if (valid > 0) gv.x = gi[gcol];
                if (valid > 1) gv.y = gi[gcol + 1];
                if (valid > 2) gv.z = gi[gcol + 2];
                if (valid > 3) gv.w = gi[gcol + 3];
            }
            a0 = fmaf(x0.x, gv.x, fmaf(x0.y, gv.y, fmaf(x0.z, gv.z, fmaf(x0.w, gv.w, a0))));
            a1 = fmaf(x1.x, gv.x, fmaf(x1.y, gv.y, fmaf(x1.z, gv.z, fmaf(x1.w, gv.w, a1))));
            a2 = fmaf(x2.x, gv.x, fmaf(x2.y, gv.y, fmaf(x2.z, gv.z, fmaf(x2.w, gv.w, a2))));
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, o);
            a1 += __shfl_xor_sync(0xffffffffu, a1, o);
            a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        }
        if (lane == 0) {
            atomicAdd(&F[3 * (int64_t)id.x + 0], -a0);
            atomicAdd(&F[3 * (int64_t)id.x + 1], -a1);
            atomicAdd(&F[3 * (int64_t)id.x + 2], -a2);
        }
        fx += a0; fy += a1; fz += a2;
        if (vir_atom) {
            const float4 r = v.ent_vec[e];
            const float q[3] = {a0, a1, a2}, rv[3] = {r.x, r.y, r.z};
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) vir[3 * a + b] -= q[a] * rv[b];
        }
    }
    if (lane == 0) {
        atomicAdd(&F[3 * i + 0], fx);
        atomicAdd(&F[3 * i + 1], fy);
        atomicAdd(&F[3 * i + 2], fz);
    }
    if (vir_atom && lane < 9) {
        float val = vir[0];
#pragma unroll
        for (int k = 1; k < 9; ++k) if (lane == k) val = vir[k];
        vir_atom[9 * i + lane] = val;
    }
}

// Balanced variants.  The grid holds as many warps as fit on the GPU at once; warp w of T
// takes the atoms whose entries fall in the w-th of T equal slices of all entries (whole
// atoms, so no atom is split), which evens out molecules of 5 and of 30 atoms and leaves no
// tail wave.  NP = passes of 32 float4 columns per entry row (W <= 128 NP): each lane decodes
// its NP column positions once, then issues all 3 NP of its loads of an entry row before any
// arithmetic, keeping about 4.6 kB per warp in flight for NP = 3.

// first atom of warp w's range: the smallest i with ent_off[i] >= ceil(w P / T); N for w = T
__device__ __forceinline__ int64_t range_start(const StoreView& v, int64_t w, int64_t T)
{
    if (w >= T) return v.N;
    const int64_t target = (w * v.P + T - 1) / T;
    int64_t lo = 0, hi = v.N;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (v.ent_off[mid] >= target) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

// per lane and pass: neighbour-species-independent part of the column map
template <int NP>
struct LaneCols {
    int loc[NP];     // radial column, or position inside an angular block
    int spc[NP];     // -1: radial block; else the second species s of block {s_j, s}
    int valid[NP];   // real columns among the four (0: padding or beyond the row)
};

template <int NP>
__device__ __forceinline__ void lane_cols(const DescDev& d, const StoreView& v, int lane, LaneCols<NP>& lc)
{
    const int W4 = v.W >> 2, A = d.n_theta * d.n_ang_r;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const int c4 = lane + 32 * p;
        const int col = 4 * c4;
        int valid;
        if (col < v.Rp) {
            lc.loc[p] = col;
            lc.spc[p] = -1;
            valid = d.n_rad - col;
        } else {
            const int ww = col - v.Rp;
            const int sp = ww / v.Ap;
            lc.loc[p] = ww - sp * v.Ap;
            lc.spc[p] = sp;
            valid = A - lc.loc[p];
        }
        valid = valid < 0 ? 0 : (valid > 4 ? 4 : valid);
        lc.valid[p] = c4 < W4 ? valid : 0;
    }
}

__device__ __forceinline__ int lane_gcol(const DescDev& d, int sj, int loc, int spc)
{
    if (spc < 0) return sj * d.n_rad + loc;
    const int a = sj < spc ? sj : spc, b = sj < spc ? spc : sj;
    return d.rad_cols + pair_block_s(a, b, d.S) * (d.n_theta * d.n_ang_r) + loc;
}

template <int NP, bool VEC>
__global__ void __launch_bounds__(kStoreWarps * 32, NP <= 3 ? 3 : 2)
k_store_adjoint_b(StoreView v, DescDev d, const float* __restrict__ g_rows, float* __restrict__ F,
                  float* __restrict__ vir_atom)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t T = (int64_t)gridDim.x * kStoreWarps;
    const int64_t w = (int64_t)blockIdx.x * kStoreWarps + warp;
    const int64_t a0 = range_start(v, w, T), a1 = range_start(v, w + 1, T);
    if (a0 >= a1) return;
    LaneCols<NP> lc;
    lane_cols<NP>(d, v, lane, lc);
    const int W4 = v.W >> 2;
    for (int64_t i = a0; i < a1; ++i) {
        const float* gi = g_rows + (size_t)v.row_of_atom[i] * d.D;
        const int64_t e0 = v.ent_off[i], e1 = v.ent_off[i + 1];
        float fx = 0.f, fy = 0.f, fz = 0.f;
        float vir[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) vir[k] = 0.f;
        for (int64_t e = e0; e < e1; ++e) {
            const int2 id = v.ent_idx[e];
            const float4* J0 = reinterpret_cast<const float4*>(v.jac + (size_t)e * 3 * v.W);
            float4 x[NP][3];
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const int c4 = lane + 32 * p;
                if (c4 < W4) {
                    x[p][0] = __ldcs(J0 + c4);
                    x[p][1] = __ldcs(J0 + W4 + c4);
                    x[p][2] = __ldcs(J0 + 2 * W4 + c4);
                } else {
                    x[p][0] = x[p][1] = x[p][2] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            float q0 = 0.f, q1 = 0.f, q2 = 0.f;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const int valid = lc.valid[p];
                float4 gv = make_float4(0.f, 0.f, 0.f, 0.f);
                if (valid > 0) {
                    const int gcol = lane_gcol(d, id.y, lc.loc[p], lc.spc[p]);
                    if (VEC) {
                        gv = *reinterpret_cast<const float4*>(gi + gcol);
                    } else {
                        gv.x = gi[gcol];
                        if (valid > 1) gv.y = gi[gcol + 1];
                        if (valid > 2) gv.z = gi[gcol + 2];
                        if (valid > 3) gv.w = gi[gcol + 3];
                    }
                }
                q0 = fmaf(x[p][0].x, gv.x, fmaf(x[p][0].y, gv.y, fmaf(x[p][0].z, gv.z, fmaf(x[p][0].w, gv.w, q0))));
                q1 = fmaf(x[p][1].x, gv.x, fmaf(x[p][1].y, gv.y, fmaf(x[p][1].z, gv.z, fmaf(x[p][1].w, gv.w, q1))));
                q2 = fmaf(x[p][2].x, gv.x, fmaf(x[p][2].y, gv.y, fmaf(x[p][2].z, gv.z, fmaf(x[p][2].w, gv.w, q2))));
            }
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
                q0 += __shfl_xor_sync(0xffffffffu, q0, o);
                q1 += __shfl_xor_sync(0xffffffffu, q1, o);
                q2 += __shfl_xor_sync(0xffffffffu, q2, o);
            }
            if (lane == 0) {
                atomicAdd(&F[3 * (int64_t)id.x + 0], -q0);
                atomicAdd(&F[3 * (int64_t)id.x + 1], -q1);
                atomicAdd(&F[3 * (int64_t)id.x + 2], -q2);
            }
            fx += q0; fy += q1; fz += q2;
            if (vir_atom) {
                const float4 r = v.ent_vec[e];
                const float q[3] = {q0, q1, q2}, rv[3] = {r.x, r.y, r.z};
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b) vir[3 * a + b] -= q[a] * rv[b];
            }
        }
        if (lane == 0 && e1 > e0) {
            atomicAdd(&F[3 * i + 0], fx);
            atomicAdd(&F[3 * i + 1], fy);
            atomicAdd(&F[3 * i + 2], fz);
        }
        if (vir_atom && lane < 9) {
            float val = vir[0];
#pragma unroll
            for (int k = 1; k < 9; ++k) if (lane == k) val = vir[k];
            vir_atom[9 * i + lane] = val;
        }
    }
}

template <int NP>
__global__ void __launch_bounds__(kStoreWarps * 32, NP <= 3 ? 3 : 2)
k_store_tangent_b(StoreView v, DescDev d, const float* __restrict__ u, float* __restrict__ wd)
{
    extern __shared__ float smf[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t T = (int64_t)gridDim.x * kStoreWarps;
    const int64_t w = (int64_t)blockIdx.x * kStoreWarps + warp;
    const int64_t a0 = range_start(v, w, T), a1 = range_start(v, w + 1, T);
    if (a0 >= a1) return;
    LaneCols<NP> lc;
    lane_cols<NP>(d, v, lane, lc);
    const int W4 = v.W >> 2, D = d.D;
    float* t = smf + (size_t)warp * ((D + 3) & ~3);
    for (int c = lane; c < D; c += 32) t[c] = 0.f;
    __syncwarp();
    for (int64_t i = a0; i < a1; ++i) {
        const float uix = u[3 * i], uiy = u[3 * i + 1], uiz = u[3 * i + 2];
        const int64_t e0 = v.ent_off[i], e1 = v.ent_off[i + 1];
        for (int64_t e = e0; e < e1; ++e) {
            const int2 id = v.ent_idx[e];
            const int64_t j = id.x;
            const float4* J0 = reinterpret_cast<const float4*>(v.jac + (size_t)e * 3 * v.W);
            float4 x[NP][3];
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const int c4 = lane + 32 * p;
                if (c4 < W4) {
                    x[p][0] = __ldcs(J0 + c4);
                    x[p][1] = __ldcs(J0 + W4 + c4);
                    x[p][2] = __ldcs(J0 + 2 * W4 + c4);
                } else {
                    x[p][0] = x[p][1] = x[p][2] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            const float vx = u[3 * j] - uix, vy = u[3 * j + 1] - uiy, vz = u[3 * j + 2] - uiz;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const int valid = lc.valid[p];
                if (valid > 0) {
                    const int gcol = lane_gcol(d, id.y, lc.loc[p], lc.spc[p]);
                    t[gcol] += fmaf(x[p][0].x, vx, fmaf(x[p][1].x, vy, x[p][2].x * vz));
                    if (valid > 1) t[gcol + 1] += fmaf(x[p][0].y, vx, fmaf(x[p][1].y, vy, x[p][2].y * vz));
                    if (valid > 2) t[gcol + 2] += fmaf(x[p][0].z, vx, fmaf(x[p][1].z, vy, x[p][2].z * vz));
                    if (valid > 3) t[gcol + 3] += fmaf(x[p][0].w, vx, fmaf(x[p][1].w, vy, x[p][2].w * vz));
                }
            }
            __syncwarp();   // the next entry may map other lanes onto these columns
        }
        float* out = wd + (size_t)v.row_of_atom[i] * D;
        for (int c = lane; c < D; c += 32) {
            out[c] = t[c];
            t[c] = 0.f;
        }
        __syncwarp();
    }
}

// resident CTAs of a kernel instance on this device, times the SM count, capped by the work
template <class K>
static unsigned balanced_blocks(K kernel, size_t smem, int64_t N)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kStoreWarps * 32, smem);
    int64_t nb = (int64_t)(sms > 0 ? sms : 1) * (per > 0 ? per : 1);
    const int64_t need = (N + kStoreWarps - 1) / kStoreWarps;
    return (unsigned)(nb < need ? nb : need);
}

template <int NP, bool VEC>
static cudaError_t store_adjoint_np(const StoreView& v, const DescDev& d, const float* g_rows, float* F,
                                    float* vir_atom, cudaStream_t s)
{
    const unsigned nb = balanced_blocks(k_store_adjoint_b<NP, VEC>, 0, v.N);
    k_store_adjoint_b<NP, VEC><<<nb, kStoreWarps * 32, 0, s>>>(v, d, g_rows, F, vir_atom);
    return cudaGetLastError();
}

template <int NP>
static cudaError_t store_tangent_np(const StoreView& v, const DescDev& d, const float* u, float* wd, cudaStream_t s)
{
    const size_t smem = (size_t)kStoreWarps * ((d.D + 3) & ~3) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_store_tangent_b<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned nb = balanced_blocks(k_store_tangent_b<NP>, smem, v.N);
    k_store_tangent_b<NP><<<nb, kStoreWarps * 32, smem, s>>>(v, d, u, wd);
    return cudaGetLastError();
}

cudaError_t launch_store_adjoint(const StoreView& v, const DescDev& d, const float* g_rows, float* F, float* vir_atom,
                                 cudaStream_t s, int* launches)
{
    const unsigned nb = (unsigned)((v.N + kStoreWarps - 1) / kStoreWarps);
    if (nb == 0) return cudaSuccess;
    const bool vec = d.n_rad % 4 == 0 && (d.n_theta * d.n_ang_r) % 4 == 0;
    const int np = (v.W / 4 + 31) / 32;
    if (np <= 6) {
        ++*launches;
        switch (np * 2 + (vec ? 1 : 0)) {
            case 2: return store_adjoint_np<1, false>(v, d, g_rows, F, vir_atom, s);
            case 3: return store_adjoint_np<1, true>(v, d, g_rows, F, vir_atom, s);
            case 4: return store_adjoint_np<2, false>(v, d, g_rows, F, vir_atom, s);
            case 5: return store_adjoint_np<2, true>(v, d, g_rows, F, vir_atom, s);
            case 6: return store_adjoint_np<3, false>(v, d, g_rows, F, vir_atom, s);
            case 7: return store_adjoint_np<3, true>(v, d, g_rows, F, vir_atom, s);
            case 8: return store_adjoint_np<4, false>(v, d, g_rows, F, vir_atom, s);
            case 9: return store_adjoint_np<4, true>(v, d, g_rows, F, vir_atom, s);
            case 10: return store_adjoint_np<5, false>(v, d, g_rows, F, vir_atom, s);
            case 11: return store_adjoint_np<5, true>(v, d, g_rows, F, vir_atom, s);
            case 12: return store_adjoint_np<6, false>(v, d, g_rows, F, vir_atom, s);
            default: return store_adjoint_np<6, true>(v, d, g_rows, F, vir_atom, s);
        }
    }
    // wider rows: one warp per atom, columns in a loop
    if (vec) k_store_adjoint<true><<<nb, kStoreWarps * 32, 0, s>>>(v, d, g_rows, F, vir_atom);
    else k_store_adjoint<false><<<nb, kStoreWarps * 32, 0, s>>>(v, d, g_rows, F, vir_atom);
    ++*launches;
    return cudaGetLastError();
}

// w_i = sum_e J_e (u_j(e) - u_i), accumulated in a shared-memory row per warp (one warp per
// atom, entries one after the other), then written as the atom's network-order row
__global__ void k_store_tangent(StoreView v, DescDev d, const float* __restrict__ u, float* __restrict__ wd)
{
    extern __shared__ float smf[];
    const int warps = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * warps + warp;
    if (i >= v.N) return;
    const int D = d.D;
    float* t = smf + (size_t)warp * ((D + 3) & ~3);
    for (int c = lane; c < D; c += 32) t[c] = 0.f;
    __syncwarp();
    const float uix = u[3 * i], uiy = u[3 * i + 1], uiz = u[3 * i + 2];
    const int64_t e0 = v.ent_off[i], e1 = v.ent_off[i + 1];
    const int W4 = v.W >> 2;
    for (int64_t e = e0; e < e1; ++e) {
        const int2 id = v.ent_idx[e];
        const int64_t j = id.x;
        const float vx = u[3 * j] - uix, vy = u[3 * j + 1] - uiy, vz = u[3 * j + 2] - uiz;
        const float4* J0 = reinterpret_cast<const float4*>(v.jac + (size_t)e * 3 * v.W);
        const float4* J1 = J0 + W4;
        const float4* J2 = J1 + W4;
        for (int c4 = lane; c4 < W4; c4 += 32) {
            const float4 x0 = __ldcs(J0 + c4), x1 = __ldcs(J1 + c4), x2 = __ldcs(J2 + c4);
            int gcol, valid;
            store_cols(d, v, id.y, c4, gcol, valid);
            const float q0 = fmaf(x0.x, vx, fmaf(x1.x, vy, x2.x * vz));
            const float q1 = fmaf(x0.y, vx, fmaf(x1.y, vy, x2.y * vz));
            const float q2 = fmaf(x0.z, vx, fmaf(x1.z, vy, x2.z * vz));
            const float q3 = fmaf(x0.w, vx, fmaf(x1.w, vy, x2.w * vz));
            if (valid > 0) t[gcol] += q0;
            if (valid > 1) t[gcol + 1] += q1;
            if (valid > 2) t[gcol + 2] += q2;
            if (valid > 3) t[gcol + 3] += q3;
        }
        __syncwarp();   // the next entry may map other lanes onto these columns
    }
    float* out = wd + (size_t)v.row_of_atom[i] * D;
    for (int c = lane; c < D; c += 32) out[c] = t[c];
}

cudaError_t launch_store_tangent(const StoreView& v, const DescDev& d, const float* u, float* wdot_rows,
                                 cudaStream_t s, int* launches)
{
    if (v.N == 0) return cudaSuccess;
    const size_t row = (size_t)((d.D + 3) & ~3) * sizeof(float);
    const int np = (v.W / 4 + 31) / 32;
    if (np <= 6 && row * kStoreWarps <= 200 * 1024) {
        ++*launches;
        switch (np) {
            case 1: return store_tangent_np<1>(v, d, u, wdot_rows, s);
            case 2: return store_tangent_np<2>(v, d, u, wdot_rows, s);
            case 3: return store_tangent_np<3>(v, d, u, wdot_rows, s);
            case 4: return store_tangent_np<4>(v, d, u, wdot_rows, s);
            case 5: return store_tangent_np<5>(v, d, u, wdot_rows, s);
            default: return store_tangent_np<6>(v, d, u, wdot_rows, s);
        }
    }
    // wider rows or descriptors: one warp per atom, columns in a loop
    int warps = (int)((200 * 1024) / row);
    warps = warps > kStoreWarps ? kStoreWarps : warps;
    if (warps < 1) return cudaErrorInvalidValue;
    const size_t smem = (size_t)warps * row;
    cudaError_t e = cudaFuncSetAttribute(k_store_tangent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned nb = (unsigned)((v.N + warps - 1) / warps);
    k_store_tangent<<<nb, warps * 32, smem, s>>>(v, d, u, wdot_rows);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace panna
