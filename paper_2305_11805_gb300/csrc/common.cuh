// Internal declarations shared by the CUDA translation units of libpanna_gb300.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/panna_gb300.h"

namespace panna {

constexpr int kMaxSpecies = 8;
constexpr int kMaxLayers = PANNA_MAX_LAYERS;

// Device status word: first error code wins; need_cap records the largest neighbour
// count seen when an atom overflowed its capacity.
struct DevStatus {
    int32_t code;
    int32_t need_cap;
    int32_t bad_index;
    int32_t stale;      // dynamics: an atom moved more than skin/2 since the neighbour build
};

__device__ __forceinline__ void set_status(DevStatus* st, int32_t code, int32_t idx)
{
    if (atomicCAS(&st->code, 0, code) == 0) st->bad_index = idx;
}

// Descriptor parameters as the kernels read them (FP32 copies plus FP64 cutoff).  The
// struct is passed by value, so the grids sit in the kernel-parameter constant bank.
constexpr int kMaxRad = 256;
constexpr int kMaxAngR = 64;
constexpr int kMaxTheta = 64;
struct DescDev {
    int32_t S, n_rad, n_ang_r, n_theta, D, n_blocks, rad_cols;
    int32_t zeta_int;      // zeta when it is an integer in [1, 4096], else 0
    float rc, rc2, eta_rad, eta_ang, zeta, eps_theta;
    float pi_rc;           // pi / rc
    double rc_d;
    float rs_rad[kMaxRad];
    float rs_ang[kMaxAngR];
    float half_cos_t[kMaxTheta];   // cos(theta_m) / 2 (float nearest)
    float half_sin_t[kMaxTheta];   // sin(theta_m) / 2
    float half_cos_lo[kMaxTheta];  // remainders: exact value - float value
    float half_sin_lo[kMaxTheta];
    float eps_theta_lo;
    float cos_half_t[kMaxTheta];   // cos(theta_m / 2), sin(theta_m / 2) (half-angle form)
    float sin_half_t[kMaxTheta];
    float zpoly[5];                // zeta log2(e) log(y) = w (c0 + c1 w^2 + ... + c4 w^8), w = t / (2 - t)
    float rs_ang_step;             // dR of a uniform angular R grid, else 0
    float cos_t[kMaxTheta], sin_t[kMaxTheta];   // cos(theta_m), sin(theta_m)
    // standard BP angular term (ang_kind 1): sector m = (lambda_m, zeta_m), shell n = eta_n
    int32_t ang_kind;              // 0 = modified (mBP), 1 = standard BP
    float bp_lambda[kMaxTheta], bp_zeta[kMaxTheta], bp_pref[kMaxTheta];   // pref = 2^(1 - zeta)
    int32_t bp_zeta_int[kMaxTheta];   // zeta when an integer in [1, 4096], else 0
    float bp_eta[kMaxAngR];
};

// Descriptor parameters (descriptor.cu): nullptr when valid, else the reason
// (*unsupported: a grid beyond the kernels' limits rather than an invalid value); and the
// DescDev of valid parameters
const char* desc_params_check(const panna_desc_params* p, bool* unsupported);
void desc_dev_from_params(const panna_desc_params* p, DescDev& d);

// Geometry of one configuration as binned on the device.
struct CfgGeom {
    double cell[9];     // rows a, b, c (identity frame for fully non-periodic configs)
    double cinv[9];     // fractional (row) = x (row) * cinv
    double lo[3];       // fractional origin of the grid
    double inv_w[3];    // 1 / fractional width of a grid cell
    int32_t n[3];       // grid cells per axis
    int32_t K[3];       // cell-offset window per axis
    int32_t per[3];     // periodic flags
    int32_t ncells;
    int64_t cell_base;  // global id of the first cell
    float sh_hi[27][3]; // image shift t.cell for t in [-1,1]^3 as hi + lo floats
    float sh_lo[27][3];
};

// Neighbour slot index packing: (t0+128) | (t1+128) << 8 | (t2+128) << 16 | species << 24
__host__ __device__ __forceinline__ int32_t pack_meta(int t0, int t1, int t2, int sp)
{
    return (t0 + 128) | ((t1 + 128) << 8) | ((t2 + 128) << 16) | (sp << 24);
}
__host__ __device__ __forceinline__ int meta_species(int32_t m) { return (m >> 24) & 0xff; }
__host__ __device__ __forceinline__ int meta_t(int32_t m, int a) { return ((m >> (8 * a)) & 0xff) - 128; }

// Workspace pointers for one call (all device memory owned by the context).
struct Work {
    int64_t N, C, cap_cells;
    int32_t cap;                 // neighbour slots per atom
    const panna_system* sys;
    DevStatus* status;
    // binning
    CfgGeom* geom;               // [C]
    int64_t* cell_count;         // [cap_cells+1]
    int64_t* cell_start;         // [cap_cells+1]
    int32_t* cell_fill;          // [cap_cells]
    int32_t* cell_atoms;         // [N]
    int32_t* atom_cell;          // [N] local cell id within the config
    int32_t* atom_cfg;           // [N]
    float4* pos_hi;              // [N] folded position, hi part
    float4* pos_lo;              // [N] lo part
    float4* pos_hi_s;            // [N] pos_hi in cell order (slot t holds atom cell_atoms[t])
    float4* pos_lo_s;            // [N] pos_lo in cell order
    int32_t* wrap;               // [N*3] integer lattice offset added by folding
    int64_t* scan_tmp;           // scan scratch
    // neighbours
    int32_t* nb_count;           // [N]
    float4* nb_vec;              // [N*cap] (dx, dy, dz, r)
    // [N*cap] low parts (dx - (float)dx, ...) of the relative vectors formed in double-float, or
    // null: written and read only for the float-pair angular terms (FP32 networks)
    float4* nb_vlo;
    int2* nb_idx;                // [N*cap] (j, meta)
    // species order
    int32_t* row_of_atom;        // [N]
    int32_t* atom_of_row;        // [N]
    int32_t* seg_off;            // [S+1] rows of species s: seg_off[s]..seg_off[s+1]-1
    int32_t* blk_counts;         // species sort scratch
    // small batches: per-split partial descriptor rows [split_rows / N][N][D] (null: no splits)
    float* split_part;
    int64_t split_rows;
};

// Small batches spread the angular pairs of one atom over several warps (descriptor and
// adjoint, blocked layout): below kSplitAtoms atoms, up to kMaxSplits warps per atom, aiming
// at kSplitTargetWarps warps in all
constexpr int64_t kSplitAtoms = 1216;
constexpr int kMaxSplits = 16;
constexpr int64_t kSplitTargetWarps = 2432;

// launch helpers implemented in the .cu files
int64_t scan_scratch_elems(int64_t n);
cudaError_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* tmp, cudaStream_t s, int* launches);
cudaError_t build_neighbors(Work& w, const DescDev& d, cudaStream_t s, int* launches);
cudaError_t species_order(Work& w, int S, cudaStream_t s, int* launches);
// Verlet list: `cand` holds the candidates of a build with cutoff rc + skin (its nb_count,
// nb_idx, cap); writes w's neighbour slots for cutoff d.rc at the current positions
cudaError_t refresh_neighbors(const Work& cand, Work& w, const DescDev& d, cudaStream_t s, int* launches);
cudaError_t export_neighbors(const Work& w, int64_t* off, int64_t* nbr_j, int32_t* shift, int64_t cap_total, cudaStream_t s, int* launches);

// descriptor family (descriptor.cu); row_map == nullptr writes row i for atom i
// acc selects the extended-precision angular evaluation (see descriptor.cu)
// variant 0: pairs by species block, 8 warps per CTA; 1: all pairs of an atom in one
// flattened range, 4 warps per CTA (full lanes for many small blocks); variant 1 falls back
// to 0 when its shared memory does not fit
cudaError_t launch_descriptor(const Work& w, const DescDev& d, float* G_rows, const int32_t* row_map, bool acc,
                              cudaStream_t s, int* launches, int variant = 0);
cudaError_t launch_adjoint(const Work& w, const DescDev& d, const float* g_rows, float* F, float* vir_atom, bool acc,
                           int variant, cudaStream_t s, int* launches);
// descriptor rows written straight into the BF16 hi (+ lo) operands of the tensor-core networks
// (compensated variants 2..4 of the modified term, batches that need no atom splits);
// cudaErrorNotSupported otherwise (then write FP32 rows and convert)
// fast: the approximate-intrinsic forms (no Newton steps, log2-based powers), enough for BF16
// networks whose operand rows hold about 16 significant bits
cudaError_t launch_descriptor_bf16(const Work& w, const DescDev& d, __nv_bfloat16* Gh, __nv_bfloat16* Gl,
                                   const int32_t* row_map, int variant, cudaStream_t s, int* launches, bool fast);
cudaError_t launch_jvp(const Work& w, const DescDev& d, const float* u, float* wdot_rows, bool acc, cudaStream_t s,
                       int* launches, int variant = 0);

// FP64 copies of the descriptor parameters (the stored Jacobians are evaluated in FP64)
struct DescGrid64 {
    double rc, eta_rad, eta_ang, zeta, eps_theta, pref;   // pref = 2^(1 - zeta)
    int32_t zeta_int;
    double rs_rad[kMaxRad];
    double rs_ang[kMaxAngR];
    double cos_t[kMaxTheta], sin_t[kMaxTheta];
};

// Stored descriptors and Jacobians of one batch (store.cu): sections of one device buffer,
// in the order and with the alignment that store_carve fixes.
constexpr int kStoreSections = 9;
struct StoreView {
    int64_t N, C, P;            // atoms, configurations, neighbour entries
    int32_t S, D, Rp, Ap, W;    // species, descriptor size, padded radial / block widths, columns
    float* G;                   // [N][D] network-order rows
    int32_t* row_of_atom;       // [N]
    int32_t* atom_of_row;       // [N]
    int32_t* seg_off;           // [S+1]
    int32_t* atom_cfg;          // [N]
    int64_t* ent_off;           // [N+1]
    int2* ent_idx;              // [P] (j, species of j)
    float4* ent_vec;            // [P] (r_e, |r_e|)
    float* jac;                 // [P][3][W]
};
// widths from the descriptor; section offsets (bytes) into off[kStoreSections] when off is
// non-null; pointers into `base` when it is non-null; returns the total size in bytes
void store_dims(const DescDev& d, StoreView& v);
int64_t store_carve(StoreView& v, char* base, int64_t* off);
// off[0..N]: exclusive scan of the neighbour counts (entry offsets of each atom)
cudaError_t launch_store_offsets(const Work& w, int64_t* off, cudaStream_t s, int* launches);
cudaError_t launch_store_entries(const Work& w, const StoreView& v, cudaStream_t s, int* launches);
cudaError_t launch_store_jacobian(const Work& w, const DescDev& d, const DescGrid64& g, const StoreView& v,
                                  cudaStream_t s, int* launches);
cudaError_t launch_store_adjoint(const StoreView& v, const DescDev& d, const float* g_rows, float* F, float* vir_atom,
                                 cudaStream_t s, int* launches);
cudaError_t launch_store_tangent(const StoreView& v, const DescDev& d, const float* u, float* wdot_rows,
                                 cudaStream_t s, int* launches);
// largest neighbour capacity and descriptor size the store kernels take
constexpr int kStoreMaxCap = 2048;
constexpr int kStoreMaxD = 49152;

// Charge equilibration (qeq.cu): per-species Gaussian widths, reference electronegativity and
// hardness, Coulomb constant; configurations of at most kQeqMax atoms
constexpr int kQeqMax = 128;
struct QeqDev { double sigma[kMaxSpecies], chi0[kMaxSpecies], hard0[kMaxSpecies]; double ke; };
size_t qeq_smem_bytes(int max_n);
// out: network outputs (rows, stride ldo, columns e, dchi, dJ); writes E_rows (row order),
// charges (atom order, may be null), adds the pair forces to F, writes the seeds
// (1, q, q^2/2) of the networks' input gradient (rows, stride lds)
cudaError_t launch_qeq(const QeqDev& qp, const Work& w, const float* out, int ldo, const double* Qtot,
                       float* E_rows, double* charges, float* F, float* seeds, int lds, cudaStream_t s,
                       int* launches);
// The charges' response for the loss gradient (see qeq.cu): inputs of the forward pass and of
// the loss; writes the reverse-pass seeds of the networks' outputs (seeds) and of their
// tangents (tr.seeds_t), and adds the charge term to *tr.loss
struct QeqTrain {
    const double* q;       // [N] charges of the forward pass
    const float* u;        // [N*3] dL/dF
    const float* odot;     // output tangents (rows, stride ldo)
    const double* alpha;   // [C] dL/dE_c
    const double* q_ref;   // [N] reference charges, or null (no charge term)
    double w_charge;
    float* seeds_t;        // rows, stride lds
    double* loss;
};
cudaError_t launch_qeq_response(const QeqDev& qp, const Work& w, const float* out, int ldo, const QeqTrain& tr,
                                float* seeds, int lds, cudaStream_t s, int* launches);

// Langevin dynamics (md.cu): per species a = (eV/A)/m in A/fs^2 and the thermal velocity
// scale sigma = sqrt(kB T a) in A/fs
struct MdSpecies { double acc[kMaxSpecies]; double sigma[kMaxSpecies]; };
cudaError_t launch_md_baoa(int64_t N, const int32_t* species, const MdSpecies& ms, double* pos, double* vel,
                           const float* F, double dt, double c1, double c2, int thermostat, uint64_t seed,
                           int64_t step, const double* pos_ref, double lim2, int32_t* stale, cudaStream_t s);
cudaError_t launch_md_b(int64_t N, const int32_t* species, const MdSpecies& ms, double* vel, const float* F,
                        double dt, cudaStream_t s);

// reductions (reduce.cu)
int cfg_chunks(int64_t N, int64_t C);
cudaError_t launch_cfg_reduce(const Work& w, const float* E_rows, const float* vir_atom, double* E_cfg, double* virial,
                              float* E_atom, double* part, cudaStream_t s, int* launches);
constexpr int kLossParts = 4 * 120;   // (energy, force) and (L1, L2) sums per block
// Loss options (Sec. II.A): term kind 0 = x^2, 1 = exp(x^2) - 1 for energies and forces,
// energies per configuration or per atom, L1/L2 penalty over the weights listed in `wr`
struct LossOpts { int e_kind, f_kind, e_per_atom; double l1, l2; };
struct ParamRanges { int n; int64_t off[kMaxSpecies * kMaxLayers]; int64_t len[kMaxSpecies * kMaxLayers]; };
// C_norm, N_norm <= 0: normalise by the batch's own counts w.C, w.N
cudaError_t launch_loss(const Work& w, int64_t C_norm, int64_t N_norm, const LossOpts& lo, const ParamRanges& wr,
                        const float* theta, const double* E_cfg, const double* E_ref, const float* F,
                        const float* F_ref, double w_force, double* loss, double* alpha_cfg, float* u, double* part,
                        cudaStream_t s, int* launches);
// dtheta += l1 sign(w) + 2 l2 w over the weights in wr
cudaError_t launch_penalty_grad(const LossOpts& lo, const ParamRanges& wr, const float* theta, float* dtheta,
                                cudaStream_t s, int* launches);
// one fused Adam step over P parameters (entries inside `frozen` keep theta, m, v)
cudaError_t launch_adam(int64_t P, float* theta, const float* g, float* m, float* v, double lr, double b1, double b2,
                        double c1, double c2, double eps, const ParamRanges& frozen, cudaStream_t s, int* launches);
cudaError_t launch_row_scale(const Work& w, const double* alpha_cfg, float* alpha_rows, cudaStream_t s, int* launches);

// message returned by panna_last_error() on this thread (api.cu)
void set_last_error_message(const char* msg);

}  // namespace panna
