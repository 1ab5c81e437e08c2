/*
 * panna_gb300.h -- C ABI of the GB300 (sm_103a) energy / force / weight-gradient path of
 * the PANNA 2.0 neural-network interatomic potential (arXiv 2305.11805).
 *
 * The method (Sec. II, II.A): every atom i gets a fixed-size descriptor G_i of its
 * environment within a cutoff rc (species-resolved Behler-Parrinello radial terms and
 * modified angular terms); a per-species multilayer perceptron (Eq. 1) maps G_i to an
 * atomic energy E_i; the total energy is sum_i E_i and forces are -dE/dx.  Training
 * matches energies and forces through a loss (Sec. II.A) whose gradient with respect to
 * the network parameters needs a second derivative through the networks.
 *
 * Conventions shared by every call
 *  - Memory: every pointer argument named "device" lives in CUDA device memory of the
 *    current device and is owned by the caller; the library never frees it.  Arguments
 *    marked "host" are host memory and are only read during the call.  The context owns
 *    its workspace (device memory grown on demand, freed by panna_destroy).
 *  - Streams: work is enqueued on the caller's stream `stream` (0 = legacy default).
 *    Unless stated otherwise a call returns after its work has completed (it ends with a
 *    stream synchronisation that also collects the device-side status word); see
 *    panna_set_async for asynchronous operation.
 *  - Errors: every call returns a panna_status and never throws across the ABI; the
 *    message of the last failure on the calling thread is in panna_last_error().  Device
 *    errors (neighbour-capacity overflow, invalid species, non-finite positions) land in
 *    a status word on the device.  On PANNA_ERR_NEIGHBOR_OVERFLOW a synchronous call
 *    has already grown its neighbour capacity and re-run once; it only fails if the
 *    retry overflows too.
 *  - Precision: positions and cells enter in FP64.  Descriptors, the descriptor adjoint
 *    (forces) and the descriptor JVP run in FP32; the networks run in FP32 or in BF16 with
 *    FP32 accumulation (mlp_precision); per-configuration energies, virials and the
 *    loss are reduced in FP64.
 *  - Units: Angstrom; energies in the units of the network output.
 */
#ifndef PANNA_GB300_H
#define PANNA_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* panna_stream_t;   /* same as cudaStream_t */

typedef enum {
    PANNA_OK = 0,
    PANNA_ERR_INVALID_ARG = 1,        /* bad sizes, null pointers, inconsistent parameters */
    PANNA_ERR_UNSUPPORTED = 2,        /* valid request outside what the kernels implement */
    PANNA_ERR_NEIGHBOR_OVERFLOW = 3,  /* an atom had more neighbours than the capacity */
    PANNA_ERR_TIMEOUT = 4,            /* a bounded device-side wait gave up */
    PANNA_ERR_CUDA = 5,               /* a CUDA runtime call failed */
    PANNA_ERR_NO_MEMORY = 6,          /* workspace allocation failed */
    PANNA_ERR_BAD_INPUT = 7           /* species out of range or non-finite coordinates */
} panna_status;

/* Activation codes (Sec. II.A: Gaussian, ReLU, tanh; linear for the output). */
enum { PANNA_ACT_LINEAR = 0, PANNA_ACT_GAUSSIAN = 1, PANNA_ACT_RELU = 2, PANNA_ACT_TANH = 3 };

/*
 * Network precision.
 *   PANNA_MLP_FP32       FP32 CUDA-core GEMMs.
 *   PANNA_MLP_BF16       tensor cores (tcgen05), BF16 operands with FP32 accumulation; every
 *                        operand is carried as a pair of BF16 numbers (hi + lo) and each
 *                        product takes three BF16 MMAs (hi*hi + hi*lo + lo*hi): about 16
 *                        significant bits per operand.
 *   PANNA_MLP_BF16_FAST  tensor cores, one BF16 rounding per operand (8 significant bits).
 * With either BF16 mode the descriptor and adjoint stay in FP32.
 */
enum { PANNA_MLP_FP32 = 0, PANNA_MLP_BF16 = 1, PANNA_MLP_BF16_FAST = 2 };

/*
 * Descriptor parameters (host memory; copied by panna_create).
 * Cutoff f_c(r) = (1 + cos(pi r / rc)) / 2 for r < rc.
 * Radial block of neighbour species s, shell n (0 <= n < n_rad):
 *     G[s*n_rad + n] = sum_j exp(-eta_rad (r_ij - rs_rad[n])^2) f_c(r_ij)
 * Angular block of the unordered species pair {s_j, s_k} (blocks in upper-triangle
 * row-major order (0,0),(0,1),..,(0,S-1),(1,1),..), entry m*n_ang_r + n:
 *     G[...] = 2^(1-zeta) sum_{j<k} max(0, 1 + cos(theta_ijk - theta_s[m]))^zeta
 *              exp(-eta_ang ((r_ij + r_ik)/2 - rs_ang[n])^2) f_c(r_ij) f_c(r_ik)
 * with cos(theta - theta_m) = cos(theta) cos(theta_m) + sin(theta) sin(theta_m) and
 * sin(theta) = sqrt(max(1 - cos^2(theta), 0) + eps_theta).
 * Size D = S*n_rad + S(S+1)/2 * n_theta * n_ang_r (Sec. III.A, III.B sizes).
 * The forms follow the standard BP / PANNA 1.0 mBP descriptors that Sec. II.A cites.
 */
/*
 * angular_kind = PANNA_ANGULAR_BP selects the standard Behler-Parrinello angular term instead
 * (the other form Sec. II.A names), in the same species-pair block layout, entry m*n_ang_r + n:
 *     G[...] = sum_{j<k} 2^(1-bp_zeta[m]) max(0, 1 + bp_lambda[m] cos(theta_ijk))^bp_zeta[m]
 *              exp(-bp_eta[n] (r_ij^2 + r_ik^2 + r_jk^2)) f_c(r_ij) f_c(r_ik) f_c(r_jk)
 * (n_theta sectors (lambda, zeta), n_ang_r shells eta; rs_ang, theta_s, eta_ang, zeta and
 * eps_theta are not read).  The BP kernels run in plain FP32 and the pair-block kernel
 * layout only (the kernel-variant knobs do not apply); stored Jacobians take mBP only.
 */
#define PANNA_ANGULAR_MBP 0
#define PANNA_ANGULAR_BP 1
typedef struct {
    int32_t n_species;      /* S, 1..8 */
    double rc;              /* cutoff (Angstrom), > 0 */
    int32_t n_rad;          /* radial shells, 1..256 */
    const double* rs_rad;   /* [n_rad] */
    double eta_rad;         /* >= 0 */
    int32_t n_ang_r;        /* angular radial shells, 1..64 */
    const double* rs_ang;   /* [n_ang_r] */
    int32_t n_theta;        /* angular sectors, 1..64 */
    const double* theta_s;  /* [n_theta] */
    double eta_ang;         /* >= 0 */
    double zeta;            /* >= 1 */
    double eps_theta;       /* >= 0 */
    int32_t angular_kind;   /* PANNA_ANGULAR_MBP (0) or PANNA_ANGULAR_BP (1) */
    const double* bp_lambda;  /* [n_theta] BP: finite */
    const double* bp_zeta;    /* [n_theta] BP: >= 1 */
    const double* bp_eta;     /* [n_ang_r] BP: >= 0 (A^-2) */
} panna_desc_params;

#define PANNA_MAX_LAYERS 8

/*
 * One species' network (Eq. 1): widths[0] = D, widths[n_layers] = 1 (an atomic energy) or 3
 * for every species (the three outputs of the charge-equilibration scheme of Sec. II.B, used
 * only by panna_qeq_energy_forces), act[l] is the activation of layer l+1.  Parameters of a species, in order for l = 1..n_layers:
 * W_l (row-major [widths[l]][widths[l-1]]) then b_l [widths[l]]; layer l computes
 * z = W_l a + b_l.  The flat parameter vector of the model is the concatenation over
 * species 0..S-1 (FP32).
 */
typedef struct {
    int32_t n_layers;
    int32_t widths[PANNA_MAX_LAYERS + 1];
    int32_t act[PANNA_MAX_LAYERS];
} panna_mlp_arch;

/*
 * A ragged batch of configurations (all device pointers, caller-owned):
 *   atom_off [n_cfg+1] int64, atoms of configuration c are atom_off[c]..atom_off[c+1]-1,
 *                     atom_off[0] = 0, atom_off[n_cfg] = n_atoms;
 *   pos      [n_atoms*3] FP64 Cartesian positions (need not be folded into the cell);
 *   species  [n_atoms] int32 in 0..S-1;
 *   cell     [n_cfg*9] FP64, rows are the lattice vectors a, b, c;
 *   pbc      [n_cfg*3] uint8 periodic flags per lattice direction;
 *   ghost    [n_atoms] uint8 or NULL.  A ghost atom (ghost[i] != 0) is a neighbour only:
 *            it is not a centre, so its atomic energy is not part of the sum of Sec. II
 *            (E_atom[i] = 0), it has an empty neighbour list and a zero descriptor row,
 *            and the force written for it is only the part -dE/dx_i that the centres of
 *            this batch exert on it.  Ghosts carry the halo of a spatial decomposition:
 *            a rank holds its own atoms plus every atom within rc of them as ghosts, and
 *            the ghost forces are summed into their owners afterwards.  NULL = no ghosts.
 * A configuration with no periodic direction ignores its cell.  Otherwise the cell must
 * be non-singular.  n_cfg and n_atoms are host values.
 */
typedef struct {
    int64_t n_cfg;
    int64_t n_atoms;
    const int64_t* atom_off;
    const double* pos;
    const int32_t* species;
    const double* cell;
    const uint8_t* pbc;
    const uint8_t* ghost;
} panna_system;

typedef struct panna_ctx panna_ctx;

/* Library version string. */
const char* panna_version(void);

/* Message of the last failure on this thread ("" if none). */
const char* panna_last_error(void);

/* D for the given parameters (Sec. III.A / III.B sizes), or -1 if they are invalid. */
int64_t panna_descriptor_size(const panna_desc_params* desc);

/*
 * Create a context bound to the current CUDA device.  `archs` (host) holds one network
 * per species (n_archs must equal desc->n_species).  Fails with PANNA_ERR_UNSUPPORTED
 * for layer widths the kernels do not implement (every width must be <= 1024, the input
 * width must equal D).
 */
panna_status panna_create(const panna_desc_params* desc, int32_t n_archs,
                          const panna_mlp_arch* archs, panna_ctx** out);

/* Release the context and its workspace (no-op for NULL). */
void panna_destroy(panna_ctx* ctx);

/* Total number of network parameters over all species (length of theta / dtheta). */
int64_t panna_param_count(const panna_ctx* ctx);

/* Per-atom neighbour capacity used by the next call (grown automatically on overflow). */
panna_status panna_set_neighbor_capacity(panna_ctx* ctx, int32_t cap);
int32_t panna_neighbor_capacity(const panna_ctx* ctx);

/*
 * async = 0 (default): every compute call synchronises `stream` at its end, checks the
 * device status word and retries once on neighbour overflow.  async = 1: calls only
 * enqueue work (no synchronisation, no retry); call panna_check afterwards.  Workspace
 * is sized on the first call for a given number of atoms, so a call with a new size is
 * never graph-capturable; repeat calls with the same sizes allocate nothing.
 */
panna_status panna_set_async(panna_ctx* ctx, int32_t async);

/*
 * With the BF16 networks (and mode 2 below) the compensated descriptor and the diagonal-order
 * adjoint use their fast forms (hardware approximations without Newton steps, y^zeta from the
 * hardware log2): about 1e-5 relative per term, below the 2^-16 of the BF16 hi + lo operand rows.
 * Arithmetic of the angular descriptor terms in kernel variants 0 and 1 (descriptor, adjoint,
 * JVP; the compensated variants 2..5 always evaluate the angle from the FP32 relative vectors,
 * t_m = 1 - y_m from the half angles and y^zeta from a series of log(1 - t): far more accurate
 * than plain FP32 at plain-FP32 cost, but the angle itself stays a single float, which the
 * zeta-th power turns into ~1e-6 relative per term, so with FP32 networks the autotuner gives
 * the descriptor only variants 0 and 1, in the extended mode below):
 *   0 = automatic (default): extended precision for the descriptor and the adjoint with FP32
 *       networks (force tolerance 1e-5 of RMS), plain FP32 with the BF16 modes (their
 *       tolerance is 1e-2) and for the JVP of the weight gradient (tolerance 1e-4);
 *   1 = extended: unit vectors, cos/sin of the angle and (1 + cos(theta - theta_m))/2
 *       carried as pairs of floats (about 4x smaller error under the zeta-th power,
 *       about twice the arithmetic);
 *   2 = plain FP32.
 */
panna_status panna_set_angular_precision(panna_ctx* ctx, int32_t mode);

/*
 * Kernel variants and the autotuner.  knob "autotune": 1 (default) = on the first
 * synchronous call for a given problem signature (atoms, configurations, neighbour
 * capacity, precision) time the candidate variants on the caller's stream (three launches
 * each) and keep the fastest; 0 = use a fixed rule (see below).
 * knobs "descriptor", "adjoint", "jvp" (the three kernels over angular pairs): -1 (default)
 * = tuned, 0 = pairs by species block (8 warps per CTA), 1 = all pairs of an atom in one
 * flattened range (4 warps per CTA; shared-memory atomics make the sums reproducible to
 * rounding rather than bit for bit), 2 / 3 / 4 = the compensated-FP32 kernels with 32 / 16 / 8
 * lanes per unit of pairs (resident warps walking the atoms; packed two-wide FP32 arithmetic;
 * the adjoint's 4 walks all units of an atom as one flattened pair range), and for the
 * adjoint only 5 = the compensated kernel walking each atom's pairs in diagonal order
 * (k, k + d mod n), whose rounds of min(32, n - 1) pairs touch distinct entries on each side,
 * so the per-entry gradients are summed without atomics in a fixed order (bit-reproducible).
 * With FP32 networks (extended angular terms) the descriptor's candidates are variants 0 and 1
 * only.  Without autotuning, batches of at least 1216 atoms take variant 2 (adjoint: 5; the
 * descriptor with FP32 networks: 0) and smaller ones variant 0
 * (several warps per atom).  knob "mlp_fp32" (PANNA_MLP_FP32 networks): a bit mask of the first layer's
 * products (descriptor width to first hidden width, almost all of the networks'
 * arithmetic) that run on the tensor cores with operands split into TF32 parts, the rest
 * staying on the CUDA cores in plain FP32: 1 = forward (three parts), 4 = tangent of the
 * weight-gradient pass (two parts), 8 = weight gradient (two parts); bit 2 (the input
 * gradient, whose forces sat at the 1e-5 bar rather than within it) is not accepted.  Default 4 | 8 = 12: the training-only products, so that energies
 * and forces are those of the plain FP32 path; the tensor cores' accumulation makes the
 * forward product about 6x less accurate than an FP32 dot product rounded to nearest.
 * 0 = everything on the CUDA cores.  Returns PANNA_ERR_INVALID_ARG for an unknown knob or
 * value.
 */
panna_status panna_set_tuning(panna_ctx* ctx, const char* knob, int32_t value);

/* The kernel variant that knob "descriptor", "adjoint" or "jvp" ran with in the last compute
 * call that used it (tuned or forced): 0 blocked, 1 flattened, 2 / 3 / 4 compensated with 32 / 16
 * / 8 lanes per (species block, theta chunk, R chunk) unit (adjoint 4: flattened units), 5
 * (adjoint only) compensated in diagonal pair order; -1 before any such call or for an unknown
 * knob. */
int32_t panna_tuning_choice(const panna_ctx* ctx, const char* knob);

/*
 * Langevin dynamics (the MD loop the paper times on a 16-atom carbon cell, Sec. III.B;
 * the paper names no integrator, read here as BAOAB, Leimkuhler and Matthews):
 *   B: v += dt/2 F/m;  A: x += dt/2 v;  O: v = c1 v + c2 sqrt(kB T / m) g;  A: x += dt/2 v;
 *   F = F(x) (panna_energy_forces arithmetic);  B: v += dt/2 F/m;
 *   c1 = exp(-friction dt), c2 = sqrt(1 - c1^2); temperature 0 and friction 0 give velocity
 *   Verlet.  g: three normals per atom and step, Box-Muller on the four 32-bit words x of
 *   Philox4x32-10 (Salmon et al., SC'11) with counter (atom low, atom high, step low, step
 *   high), key (seed low, seed high), uniforms (x + 1/2) 2^-32; the atom index is the
 *   global one of the batch, the step index step0 + t.
 * Every configuration of the batch follows its own trajectory.  Units: A, fs, amu, eV, K
 * (1 eV/A on 1 amu = 9.648533212e-3 A/fs^2, kB = 8.617333262e-5 eV/K).
 * Neighbour-list reuse: the neighbour search runs with cutoff rc + skin and is repeated
 * only when some atom has moved more than skin/2 since the last search (skin 0: every step);
 * in between, the stored candidates are re-tested at the current positions with the full
 * search's arithmetic, so the neighbour sets are those of a fresh search.
 */
typedef struct {
    double dt;             /* time step, fs */
    double temperature;    /* K */
    double friction;       /* 1/fs */
    double skin;           /* A */
    const double* mass;    /* [n_species] amu, host */
    uint64_t seed;         /* key of the noise stream */
    int64_t step0;         /* step index of the first step (counter of the noise stream) */
} panna_md_params;

/*
 * n_steps of the dynamics above.  sys->pos (device, FP64) is moved in place; vel
 * [n_atoms*3] FP64 device, A/fs, in/out; F [n_atoms*3] FP32 device in/out: the forces at the
 * current positions on entry if forces_valid != 0 (else computed first), at the final
 * positions on exit; E_cfg [n_cfg] FP64 device out: energies at the final positions;
 * E_traj [n_steps*n_cfg] FP64 device (may be NULL): energies after every step; *n_builds
 * (host, may be NULL): neighbour searches done.  Synchronous (one small status read per
 * step).  A neighbour-capacity overflow during the run returns PANNA_ERR_NEIGHBOR_OVERFLOW
 * with positions and velocities advanced to that step (raise the capacity and restart from
 * a copy); ghost atoms are rejected (PANNA_ERR_UNSUPPORTED).
 */
panna_status panna_md_run(panna_ctx* ctx, const panna_system* sys, double* vel, const float* theta,
                          int32_t mlp_precision, const panna_md_params* params, int64_t n_steps,
                          float* F, int32_t forces_valid, double* E_cfg, double* E_traj,
                          int64_t* n_builds, panna_stream_t stream);

/*
 * Normalisers of the training loss (Sec. II.A): with n_cfg_total > 0 and n_atoms_total > 0,
 * panna_loss_grad divides the energy term by n_cfg_total and the force term by
 * 3 * n_atoms_total instead of the batch's own counts.  In data-parallel training each
 * rank passes the global counts, so that the ranks' losses and gradients add up (one
 * all-reduce) to those of the whole global batch.  (0, 0) restores the default; any other
 * non-positive value is PANNA_ERR_INVALID_ARG.
 */
panna_status panna_set_loss_normalization(panna_ctx* ctx, int64_t n_cfg_total, int64_t n_atoms_total);

/*
 * Loss options of Sec. II.A (the paper names the choices; the exponential form is read as
 * exp(x^2) - 1, equal to the quadratic to leading order):
 *   L = (1/C) sum_c l_E(d_c) + w_force/(3N) sum_{m,a} l_F(F_ma - F_ref_ma)
 *       + l1 sum |w| + l2 sum w^2,
 * l(x) = x^2 (PANNA_LOSS_QUADRATIC) or exp(x^2) - 1 (PANNA_LOSS_EXPONENTIAL),
 * d_c = E_c - E_ref_c, or (E_c - E_ref_c) / n_c with energy_per_atom, the penalty over every
 * weight of every layer and species (biases excluded; the sign of 0 is 0).  Applies to
 * panna_loss_grad.  NULL restores the default (quadratic, per configuration, no penalty).
 * The exponential terms suit small residuals (per-atom energies, a trained model).
 */
#define PANNA_LOSS_QUADRATIC 0
#define PANNA_LOSS_EXPONENTIAL 1
typedef struct {
    int32_t energy_loss;
    int32_t force_loss;
    int32_t energy_per_atom;
    double l1;
    double l2;
} panna_loss_options;
panna_status panna_set_loss_options(panna_ctx* ctx, const panna_loss_options* options);

/*
 * Adam (Sec. II.A; Kingma and Ba, Algorithm 1) on the flat parameter vector, one fused pass:
 *   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
 *   theta -= lr_t (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps),
 *   lr_t = lr decay_rate^(t / decay_steps) (exponential decay; decay_steps 0: constant).
 * theta, grad, m, v: [P] FP32 device (m, v zero before step t = 1); t >= 1.  Parameters of
 * layers frozen with panna_set_frozen keep theta, m and v (fine tuning, transfer learning).
 * Asynchronous on `stream`.
 */
typedef struct {
    double lr;
    double beta1;
    double beta2;
    double eps;
    double decay_rate;
    double decay_steps;
} panna_adam_params;
panna_status panna_adam_step(panna_ctx* ctx, float* theta, const float* grad, float* m, float* v, int64_t t,
                             const panna_adam_params* params, panna_stream_t stream);

/* Freeze (frozen != 0) or release the weights and biases of layer `layer` (0 = first) of
 * species `species` for panna_adam_step. */
panna_status panna_set_frozen(panna_ctx* ctx, int32_t species, int32_t layer, int32_t frozen);

/* Synchronise `stream` and return (and clear) the device status word. */
panna_status panna_check(panna_ctx* ctx, panna_stream_t stream);

/*
 * Neighbour list (Sec. I locality, cutoff rc): every entry (i, j, n) with
 * 0 < |x_j + n.cell - x_i| < rc, j != i or n != 0, including periodic self-images and
 * several images of one atom in cells narrower than 2 rc.  Output in CSR form (device):
 *   nbr_off [n_atoms+1] int64, entries of atom i at nbr_off[i]..nbr_off[i+1]-1,
 *   nbr_j   [cap_total] int64 (global atom index), nbr_shift [cap_total*3] int32 (n).
 * Within an atom the entries are grouped by neighbour species (ascending), in a fixed
 * deterministic order inside a group.  *n_total (host) receives the number of entries;
 * if it exceeds cap_total nothing is written past cap_total and the call returns
 * PANNA_ERR_INVALID_ARG.  Always synchronous.
 */
panna_status panna_neighbors(panna_ctx* ctx, const panna_system* sys, int64_t cap_total,
                             int64_t* nbr_off, int64_t* nbr_j, int32_t* nbr_shift,
                             int64_t* n_total, panna_stream_t stream);

/* Descriptors G [n_atoms*D] FP32 (device, row i = atom i).  Sec. II.A. */
panna_status panna_descriptors(panna_ctx* ctx, const panna_system* sys, float* G,
                               panna_stream_t stream);

/*
 * Energies and forces (Sec. II): theta [P] FP32 device parameters (layout above).
 *   E_cfg  [n_cfg] FP64 per-configuration energy (device, required)
 *   E_atom [n_atoms] FP32 atomic energies (device, may be NULL)
 *   F      [n_atoms*3] FP32 forces -dE/dx (device, required)
 *   virial [n_cfg*9] FP64, W_ab = -sum over neighbour entries q_a r_b with
 *          q = dE_i/dr_ij (device, may be NULL)
 * mlp_precision: PANNA_MLP_FP32, PANNA_MLP_BF16 or PANNA_MLP_BF16_FAST (see above); the BF16
 * modes need at least one hidden layer and a descriptor size that is a multiple of 8.
 */
panna_status panna_energy_forces(panna_ctx* ctx, const panna_system* sys, const float* theta,
                                 int32_t mlp_precision, double* E_cfg, float* E_atom, float* F,
                                 double* virial, panna_stream_t stream);

/*
 * Vector-Jacobian product of (E_cfg, F) with respect to the parameters: given upstream
 * gradients dE [n_cfg] FP64 and dF [n_atoms*3] FP32 (either may be NULL = zero), writes
 *   dtheta [P] FP32 = sum_c dE_c dE_c/dtheta + sum_{m,a} dF_ma dF_ma/dtheta.
 * The force part is the double backward through the networks: with u = dF,
 * w_i = sum_e dG_i/dr_e (u_j(e) - u_i) (descriptor JVP) and g_i = dE_i/dG_i,
 * dtheta += -d/dtheta sum_i g_i . w_i.  Descriptors are recomputed, never stored with
 * their Jacobians (Sec. II.A, on-the-fly descriptors).  FP32 networks only.  With ghost
 * atoms the sums run over the non-ghost centres, and dF must hold, on each ghost, the
 * upstream gradient of the atom it stands for (the products then add up over ranks).
 */
panna_status panna_param_vjp(panna_ctx* ctx, const panna_system* sys, const float* theta,
                             const double* dE, const float* dF, float* dtheta,
                             panna_stream_t stream);

/*
 * One training step's loss and parameter gradient (Sec. II.A: quadratic energy and force
 * terms with a relative factor, energy per configuration, force per component):
 *   L = (1/C) sum_c (E_c - E_ref_c)^2 + w_force/(3N) sum_{m,a} (F_ma - F_ref_ma)^2
 * E_ref [n_cfg] FP64 and F_ref [n_atoms*3] FP32 device inputs; outputs (device):
 *   loss [1] FP64, dtheta [P] FP32 = dL/dtheta, and optionally E_cfg [n_cfg] FP64 and
 *   F [n_atoms*3] FP32 (may be NULL).  FP32 networks only.  C and N are the batch's own
 * counts unless panna_set_loss_normalization gave others.  A batch with ghost atoms is
 * rejected (PANNA_ERR_UNSUPPORTED): its ghost forces are partial sums.
 */
panna_status panna_loss_grad(panna_ctx* ctx, const panna_system* sys, const float* theta,
                             const double* E_ref, const float* F_ref, double w_force,
                             double* loss, float* dtheta, double* E_cfg, float* F,
                             panna_stream_t stream);

/*
 * Long-range electrostatics by charge equilibration (Sec. II.B).  The networks have three
 * outputs per atom (created with widths[n_layers] = 3): a local energy e_i and corrections to
 * the electronegativity and hardness of the atom's species, chi_i = chi0[s] + out_1 and
 * J_i = hard0[s] + out_2 (the second-order expansion of the energy in the atomic charge).
 * The paper defers the electrostatic form to its reference; this library takes Gaussian
 * charge distributions of per-species width sigma[s]:
 *     E_c = sum_i (e_i + chi_i q_i + J_i q_i^2 / 2) + 1/2 sum_ij q_i q_j K_ij,
 *     K_ij = k erf(r_ij / g_ij) / r_ij, g_ij = sqrt(2 (sigma_i^2 + sigma_j^2)),
 *     K_ii = k / (sigma_i sqrt(pi)),
 * and the charges q of each configuration are the stationary point of E_c under
 * sum_i q_i = Q_c (the linear system [A 1; 1^T 0][q; lam] = [-chi; Q_c], A = diag(J) + K,
 * solved in FP64 with partial pivoting; erf and exp of the pair terms in FP32).  Forces are
 * -dE_c/dx at those charges.  Direct
 * sums over all pairs of a configuration: non-periodic configurations of at most 128 atoms
 * (clusters, molecules; PANNA_ERR_UNSUPPORTED otherwise).  Units: A, e, eV;
 * k_coulomb = 0 selects 14.399645478425668 eV A / e^2.
 */
typedef struct {
    const double* sigma;   /* [n_species] Gaussian charge widths (A), > 0, host */
    const double* chi0;    /* [n_species] reference electronegativities (eV / e), host */
    const double* hard0;   /* [n_species] reference hardnesses (eV / e^2), host */
    double k_coulomb;      /* eV A / e^2; 0 = the SI value */
} panna_qeq_params;

/* Set the constants above (copied); the context's networks must have 3 outputs. */
panna_status panna_set_qeq(panna_ctx* ctx, const panna_qeq_params* params);

/*
 * Energies, charges and forces with charge equilibration.  total_charge [n_cfg] FP64 device
 * (NULL = neutral configurations); outputs (device): E_cfg [n_cfg] FP64, E_atom [n_atoms]
 * FP32 (may be NULL; E_atom_i = e_i + chi_i q_i + J_i q_i^2/2 + q_i (K q)_i / 2), charges
 * [n_atoms] FP64 (may be NULL), F [n_atoms*3] FP32.  FP32 networks.  A singular system
 * returns PANNA_ERR_BAD_INPUT naming the configuration.  Follows panna_set_async like the
 * other compute calls; with profiling on, the stages are "neighbors", "descriptor", "mlp"
 * (forward), "forces" (the charge solve, energies and pair forces), "adjoint" (input
 * gradient and descriptor adjoint) and "loss" (per-configuration sums).
 */
panna_status panna_qeq_energy_forces(panna_ctx* ctx, const panna_system* sys, const float* theta,
                                     const double* total_charge, double* E_cfg, float* E_atom,
                                     double* charges, float* F, panna_stream_t stream);

/*
 * Training through the charge-equilibration layer (Sec. II.B: reference charges may enter the
 * loss or be left out).  Loss = the panna_loss_grad loss of the equilibrated energies and
 * forces (same options and normalisers) + w_charge sum_i (q_i - q_ref_i)^2 when q_ref
 * [n_atoms] FP64 device is given (NULL: no charge term).  dtheta [P] FP32 = dL/dtheta: the
 * energy part at fixed charges (their response cancels at the constrained stationary point),
 * the force part by the double backward with output seeds (1, q_i, q_i^2/2), and the charges'
 * response dq/dtheta, which the force and charge terms need, from one more solve with the same
 * matrix.  Outputs as panna_loss_grad, plus the charges [n_atoms] FP64 (may be NULL).  FP32
 * networks on the CUDA cores.
 */
panna_status panna_qeq_loss_grad(panna_ctx* ctx, const panna_system* sys, const float* theta,
                                 const double* total_charge, const double* E_ref, const float* F_ref,
                                 double w_force, const double* q_ref, double w_charge, double* loss,
                                 float* dtheta, double* E_cfg, double* charges, float* F,
                                 panna_stream_t stream);

/*
 * Precomputed descriptors with stored Jacobians (Sec. II.A: descriptors can be computed
 * once for a whole dataset and reused in every epoch, with their derivatives stored for the
 * forces, at the price of the memory that takes; the default path recomputes them in every
 * call).  A store holds one batch; on a GPU with 288 GB of HBM a dataset of many batches can
 * stay resident, and a training step then streams the stored Jacobians instead of
 * recomputing the angular terms.
 *
 * Use: panna_store_plan (neighbour search, sizes) -> allocate info.bytes of device memory,
 * 256-byte aligned -> panna_store_build -> any number of panna_store_energy_forces /
 * panna_store_loss_grad calls with that batch's panna_system (only n_cfg, n_atoms and
 * atom_off are read; the other pointers may be NULL) and any parameters theta.
 *
 * Binary format of a store (a documented layout, so that descriptors and derivatives made
 * by other programs can be used): nine sections, each starting at the next multiple of 256
 * bytes from the buffer start (panna_store_sections returns the byte offsets), in order:
 *   0 G           float32 [n_atoms][D]     descriptor rows in network order: rows of species s
 *                                          are seg_off[s]..seg_off[s+1]-1, row r is atom
 *                                          atom_of_row[r]
 *   1 row_of_atom int32   [n_atoms]
 *   2 atom_of_row int32   [n_atoms]
 *   3 seg_off     int32   [S+1]
 *   4 atom_cfg    int32   [n_atoms]        configuration of each atom
 *   5 ent_off     int64   [n_atoms+1]      neighbour entries of atom i: ent_off[i]..ent_off[i+1]-1
 *   6 ent_idx     int32   [n_entries][2]   (j, species of j) of entry e = (i, j, n)
 *   7 ent_vec     float32 [n_entries][4]   (r_e = x_j + n.cell - x_i, |r_e|)
 *   8 jac         float32 [n_entries][3][width]: jac[e][a][c] = d G_i[col(c)] / d r_e[a], where
 *                 with Rp = 4 ceil(n_rad/4), A = n_theta n_ang_r, Ap = 4 ceil(A/4),
 *                 width = Rp + S Ap, s_j the neighbour's species:
 *                   c < Rp:              col = s_j n_rad + c                   (c < n_rad)
 *                   c = Rp + s Ap + l:   col = S n_rad + blk(min(s_j,s), max(s_j,s)) A + l  (l < A)
 *                 blk(a, b) the upper-triangle block index of the descriptor layout; the
 *                 padding columns (c >= n_rad below Rp, l >= A) hold zeros.  All other
 *                 columns of dG_i/dr_e are zero by the descriptor's definition.
 * The library's build evaluates J in FP64 and rounds it to FP32; G is the FP32 descriptor of
 * panna_descriptors.  Stores take batches without ghost atoms, D <= 49152 and at most 2048
 * neighbours per atom (PANNA_ERR_UNSUPPORTED otherwise).  The evaluation calls check the
 * sizes of a store but not its contents: a store written by another program must hold
 * indices in range (j < n_atoms, species < S, offsets within the sections).
 */
typedef struct {
    int64_t n_atoms;     /* batch the store was planned for */
    int64_t n_cfg;
    int64_t n_entries;   /* neighbour entries (i, j, n) */
    int32_t D;           /* descriptor size */
    int32_t width;       /* Jacobian columns per entry and Cartesian component */
    int64_t bytes;       /* device bytes of the store */
} panna_store_info;

/* Neighbour search of `sys` and the store's sizes into *info (host).  Synchronous. */
panna_status panna_store_plan(panna_ctx* ctx, const panna_system* sys, panna_store_info* info,
                              panna_stream_t stream);

/* Byte offsets of the nine sections above for a planned store: offsets[9] (host). */
panna_status panna_store_sections(const panna_ctx* ctx, const panna_store_info* info, int64_t* offsets);

/*
 * Fill `store` (device, info->bytes, 256-byte aligned, caller-owned) for the batch `sys` that
 * was planned (its positions must give the same number of neighbour entries, else
 * PANNA_ERR_INVALID_ARG).  Synchronous.
 */
panna_status panna_store_build(panna_ctx* ctx, const panna_system* sys, const panna_store_info* info,
                               void* store, panna_stream_t stream);

/* panna_energy_forces from a store (same outputs, same precisions). */
panna_status panna_store_energy_forces(panna_ctx* ctx, const panna_system* sys, const panna_store_info* info,
                                       const void* store, const float* theta, int32_t mlp_precision,
                                       double* E_cfg, float* E_atom, float* F, double* virial,
                                       panna_stream_t stream);

/*
 * panna_loss_grad from a store (same loss, options, normalisers and outputs).  The force
 * part of the gradient takes the descriptor tangent w_i = sum_e J_e (u_j(e) - u_i) from the
 * stored Jacobians.
 */
panna_status panna_store_loss_grad(panna_ctx* ctx, const panna_system* sys, const panna_store_info* info,
                                   const void* store, const float* theta, const double* E_ref,
                                   const float* F_ref, double w_force, double* loss, float* dtheta,
                                   double* E_cfg, float* F, panna_stream_t stream);

/*
 * CUDA-graph form of panna_energy_forces for repeated evaluation of one ragged batch (the
 * same device arrays, contents updated in place, e.g. positions in an MD loop):
 * panna_capture runs the call once synchronously (sizing the workspace, tuning kernel
 * variants, checking the status word), then records the same sequence of kernel launches
 * into a CUDA graph owned by the context (on `stream`, or on an internal stream when
 * `stream` is the legacy default stream).  panna_replay launches that graph on `stream`
 * without any host synchronisation; call panna_check afterwards to read the device status
 * word (a neighbour-capacity overflow inside a replay is reported there, not retried).
 * The graph keeps the pointers given to panna_capture; a new capture replaces the old one.
 */
panna_status panna_capture(panna_ctx* ctx, const panna_system* sys, const float* theta, int32_t mlp_precision,
                           double* E_cfg, float* E_atom, float* F, double* virial, panna_stream_t stream);
panna_status panna_replay(panna_ctx* ctx, panna_stream_t stream);

/*
 * Number of kernels the last compute call launched (for launch accounting), and the
 * device time of the named stage of the last call in milliseconds when profiling is on
 * (panna_set_profiling(ctx, 1) records CUDA events around each stage on `stream`).
 * Stages: "neighbors", "descriptor", "mlp", "adjoint", "forces", "jvp", "mlp_grad",
 * "loss".  Returns -1 for an unknown stage or when profiling is off.
 */
int32_t panna_last_launch_count(const panna_ctx* ctx);
panna_status panna_set_profiling(panna_ctx* ctx, int32_t on);
float panna_stage_ms(const panna_ctx* ctx, const char* stage);

/*
 * Measured throughput of the arithmetic units that bound the descriptor, adjoint and JVP
 * kernels (they perform hundreds of FP32 operations per byte they move, so their roofline is
 * an arithmetic one, not HBM): *fp32_tflops (host) = FP32 FMA throughput in TFLOP/s (an FMA
 * counts as two operations), *ex2_gops (host) = multi-function-unit ex2 results per second in
 * units of 1e9.  Microbenchmark kernels with independent dependency chains on every SM, timed
 * with CUDA events on `stream` (best of three launches after a warm-up, about 0.2 s in all),
 * at whatever clocks the GPU runs at the time.  Allocates and frees a few kB (stream-ordered).
 * The paper has no counterpart: this is the denominator of the kernels' reported efficiency.
 */
panna_status panna_measure_alu_peaks(double* fp32_tflops, double* ex2_gops, panna_stream_t stream);

/* As panna_measure_alu_peaks, plus *fp32x2_tflops (host): the same FMA chains issued as packed
 * two-wide FP32 FMAs (one instruction per two FMAs), which the angular kernels use. */
panna_status panna_measure_alu_peaks2(double* fp32_tflops, double* fp32x2_tflops, double* ex2_gops,
                                      panna_stream_t stream);

/*
 * Descriptors G [n_atoms*D] FP32 (device, row i = atom i) of a small batch, computed
 * without allocating any memory: no context, no cudaMalloc, no cudaFree.  The paper has
 * no counterpart; this entry point exists for callers that cannot allocate device memory
 * -- a host program whose memory pool already owns all of the GPU's memory, or a callback
 * (such as a force call from inside another code's time step) in which new device
 * allocations are not allowed.  Same parameters and result as panna_descriptors.
 *
 * Scratch (cell lists, neighbour lists, a status word) lives in one static device array
 * of 32 MiB that every GPU which loads this library holds until the process exits.  It
 * takes about 100 bytes per atom and 900 per configuration for binning, plus 24 bytes per
 * neighbour slot (at most 256 slots per atom, as many as fit): roughly 20,000 atoms with
 * 64 neighbours each.  A batch that does not leave room for 8 slots per atom is rejected
 * with PANNA_ERR_INVALID_ARG before any work; an atom with more neighbours than the slots
 * that fit gives PANNA_ERR_NEIGHBOR_OVERFLOW.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture.  Every call uses the same array and clears what must start at
 * zero: calls that overlap on the GPU (other streams, other host threads) race.  The call
 * synchronises `stream`; errors are also reported through panna_last_error().
 */
panna_status panna_descriptors_static(const panna_desc_params* desc, const panna_system* sys, float* G,
                                      panna_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* PANNA_GB300_H */
