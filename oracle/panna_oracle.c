/*
 * FP64 CPU oracle for the PANNA 2.0 energy/force/weight-gradient hot path
 * (arXiv 2305.11805).  TEST INFRASTRUCTURE ONLY: tests, the smoke check and the
 * benchmark's CPU-baseline leg call it; the product path never does.  It shares no
 * code, header, table or helper with the CUDA library.
 *
 * Plain, slow, obviously correct: brute force over every atom pair and every
 * periodic image, one centre atom at a time, everything in double precision,
 * single thread.
 *
 * What is computed, and where it comes from:
 *  - total energy as a sum of atomic energies, each a function of the atom's
 *    local environment within the cutoff (Sec. I, Sec. II);
 *  - the species-resolved Behler-Parrinello radial and modified (mBP) angular
 *    descriptors (Sec. II.A: the paper defers the formulas to BP and PANNA 1.0; the
 *    reading taken here is spelled out at orc_center below);
 *  - per-species multilayer perceptrons, a^l = sigma(W^l a^(l-1) + b^l) (Eq. 1) with
 *    Gaussian / ReLU / tanh / linear activations (Sec. II.A);
 *  - forces as minus the derivative of the energy with respect to positions (Sec. II);
 *  - virial W_ab = -sum over neighbour entries of q_a r_b, q = dE_i/dr_ij;
 *  - loss = energy term + weighted force term, quadratic, energy per configuration,
 *    force per component (Sec. II.A), and its exact gradient with respect to all
 *    network parameters.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXL 8

typedef struct {
    int n_species;
    double rc;
    int n_rad;
    const double* rs_rad;
    double eta_rad;
    int n_ang_r;
    const double* rs_ang;
    int n_theta;
    const double* theta_s;
    double eta_ang;
    double zeta;
    double eps_theta;
    int angular_kind;          /* 0: modified angular term (mBP), 1: standard BP term */
    const double* bp_lambda;   /* [n_theta] BP: lambda_m */
    const double* bp_zeta;     /* [n_theta] BP: zeta_m */
    const double* bp_eta;      /* [n_ang_r] BP: eta_n */
} orc_desc;

/* Network of one species: n_layers, widths[0..n_layers] (widths[0] = D, last = 1),
 * act[0..n_layers-1] with 0 linear, 1 Gaussian exp(-x^2), 2 ReLU, 3 tanh.
 * Parameters: per layer W (row-major [out][in]) then b [out]. */
typedef struct {
    int n_layers;
    int widths[ORC_MAXL + 1];
    int act[ORC_MAXL];
} orc_arch;

int orc_descriptor_size(const orc_desc* p)
{
    int s = p->n_species;
    return s * p->n_rad + s * (s + 1) / 2 * p->n_theta * p->n_ang_r;
}

/* Index of the unordered species pair (a <= b) in row-major upper-triangle order. */
static int pair_block(int a, int b, int S)
{
    if (a > b) { int t = a; a = b; b = t; }
    return a * S - a * (a - 1) / 2 + (b - a);
}

/* smooth cosine cutoff and its derivative */
static double fcut(double r, double rc) { return r < rc ? 0.5 * (1.0 + cos(M_PI * r / rc)) : 0.0; }
static double dfcut(double r, double rc) { return r < rc ? -0.5 * M_PI / rc * sin(M_PI * r / rc) : 0.0; }

/* ------------------------------------------------------------------------- */
/* geometry                                                                   */
/* ------------------------------------------------------------------------- */

static void inv3(const double* m, double* inv)
{
    double det = m[0] * (m[4] * m[8] - m[5] * m[7]) - m[1] * (m[3] * m[8] - m[5] * m[6])
               + m[2] * (m[3] * m[7] - m[4] * m[6]);
    inv[0] = (m[4] * m[8] - m[5] * m[7]) / det;
    inv[1] = (m[2] * m[7] - m[1] * m[8]) / det;
    inv[2] = (m[1] * m[5] - m[2] * m[4]) / det;
    inv[3] = (m[5] * m[6] - m[3] * m[8]) / det;
    inv[4] = (m[0] * m[8] - m[2] * m[6]) / det;
    inv[5] = (m[2] * m[3] - m[0] * m[5]) / det;
    inv[6] = (m[3] * m[7] - m[4] * m[6]) / det;
    inv[7] = (m[1] * m[6] - m[0] * m[7]) / det;
    inv[8] = (m[0] * m[4] - m[1] * m[3]) / det;
}

/* For each periodic direction a: how many images either side must be scanned so that
 * every (j, n) with |x_j + n.cell - x_i| < radius is visited, given that both atoms'
 * fractional coordinates were first folded into [0,1).  The fractional difference of
 * folded atoms is in (-1,1) and a displacement of length d changes fractional
 * coordinate a by at most d / h_a (h_a = cell width perpendicular to the other two
 * lattice vectors), so |n'_a| <= radius/h_a + 1 suffices. */
static void image_window(const double* cell, const uint8_t* pbc, double radius, int* K)
{
    const double* a = cell; const double* b = cell + 3; const double* c = cell + 6;
    double bxc[3] = {b[1] * c[2] - b[2] * c[1], b[2] * c[0] - b[0] * c[2], b[0] * c[1] - b[1] * c[0]};
    double cxa[3] = {c[1] * a[2] - c[2] * a[1], c[2] * a[0] - c[0] * a[2], c[0] * a[1] - c[1] * a[0]};
    double axb[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
    double vol = fabs(a[0] * bxc[0] + a[1] * bxc[1] + a[2] * bxc[2]);
    double h[3];
    h[0] = vol / sqrt(bxc[0] * bxc[0] + bxc[1] * bxc[1] + bxc[2] * bxc[2]);
    h[1] = vol / sqrt(cxa[0] * cxa[0] + cxa[1] * cxa[1] + cxa[2] * cxa[2]);
    h[2] = vol / sqrt(axb[0] * axb[0] + axb[1] * axb[1] + axb[2] * axb[2]);
    for (int d = 0; d < 3; ++d) K[d] = pbc[d] ? (int)ceil(radius / h[d]) + 1 : 0;
}

/* integer lattice offset that folds x into the cell (periodic directions only) */
static void fold_offset(const double* x, const double* cinv, const uint8_t* pbc, int* m)
{
    for (int d = 0; d < 3; ++d) {
        double s = x[0] * cinv[0 * 3 + d] + x[1] * cinv[1 * 3 + d] + x[2] * cinv[2 * 3 + d];
        m[d] = pbc[d] ? -(int)floor(s) : 0;
    }
}

typedef struct {
    int32_t j;        /* neighbour atom (index within the configuration) */
    int32_t n[3];     /* image: r = x_j + n.cell - x_i */
    double r[3];      /* relative vector */
    int32_t sp;       /* species of j */
} orc_nb;

/* All entries (j, n) with 0 < |x_j + n.cell - x_i| < radius, in lexicographic order of
 * (j, n0, n1, n2); entry (i, 0) excluded.  Candidates are restricted to the atom list
 * `cand` (all atoms of the configuration when cand == NULL).  Returns the count; at
 * most `cap` entries are written. */
static int64_t neighbours_of(int64_t i, int64_t n, const double* pos, const int32_t* spec,
                             const double* cell, const uint8_t* pbc, double radius,
                             const int64_t* cand, int64_t n_cand, int64_t cap, orc_nb* out)
{
    double cinv[9];
    int K[3] = {0, 0, 0};
    int mi[3] = {0, 0, 0};
    int periodic = pbc[0] || pbc[1] || pbc[2];
    if (periodic) {
        inv3(cell, cinv);
        image_window(cell, pbc, radius, K);
        fold_offset(pos + 3 * i, cinv, pbc, mi);
    }
    int64_t cnt = 0;
    int64_t nc = cand ? n_cand : n;
    for (int64_t q = 0; q < nc; ++q) {
        int64_t j = cand ? cand[q] : q;
        int mj[3] = {0, 0, 0};
        if (periodic) fold_offset(pos + 3 * j, cinv, pbc, mj);
        for (int a = -K[0]; a <= K[0]; ++a)
        for (int b = -K[1]; b <= K[1]; ++b)
        for (int c = -K[2]; c <= K[2]; ++c) {
            int nn[3] = {a + mj[0] - mi[0], b + mj[1] - mi[1], c + mj[2] - mi[2]};
            if (j == i && nn[0] == 0 && nn[1] == 0 && nn[2] == 0) continue;
            double r[3];
            for (int d = 0; d < 3; ++d)
                r[d] = pos[3 * j + d] + nn[0] * cell[0 + d] + nn[1] * cell[3 + d] + nn[2] * cell[6 + d]
                       - pos[3 * i + d];
            double rr = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
            if (rr < radius) {
                if (cnt < cap) {
                    out[cnt].j = (int32_t)j;
                    memcpy(out[cnt].n, nn, sizeof nn);
                    memcpy(out[cnt].r, r, sizeof r);
                    out[cnt].sp = spec ? spec[j] : 0;
                }
                ++cnt;
            }
        }
    }
    return cnt;
}

static int cmp_nb(const void* pa, const void* pb)
{
    const orc_nb* a = (const orc_nb*)pa; const orc_nb* b = (const orc_nb*)pb;
    if (a->j != b->j) return a->j < b->j ? -1 : 1;
    for (int d = 0; d < 3; ++d) if (a->n[d] != b->n[d]) return a->n[d] < b->n[d] ? -1 : 1;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* descriptor of one centre atom and its Jacobian                             */
/* ------------------------------------------------------------------------- */

/*
 * G and (optionally) J = dG/dr for one centre atom with neighbour entries nb[0..nnb).
 *
 * Reading of the BP / mBP descriptor (the paper cites the forms, Sec. II.A; the sizes
 * it prints in Sec. III.A and III.B fix the species-resolved layout):
 *   f_c(r) = (1 + cos(pi r / rc)) / 2 for r < rc, else 0.
 *   Radial, block of neighbour species s (species order), shells n inner:
 *     G[s*n_rad + n] = sum_{j: s_j = s} exp(-eta_rad (r_ij - Rs_n)^2) f_c(r_ij)
 *   Angular, block of the unordered species pair {s_j, s_k} (upper-triangle row-major
 *   order), index m*n_ang_r + n inside the block, every unordered pair of distinct
 *   neighbour entries j < k counted once:
 *     G[...] += 2^(1-zeta) max(0, 1 + cos(theta_ijk - theta_m))^zeta
 *               * exp(-eta_ang ((r_ij + r_ik)/2 - R_n)^2) f_c(r_ij) f_c(r_ik)
 *   with cos(theta - theta_m) = cos(theta) cos(theta_m) + sin(theta) sin(theta_m),
 *   cos(theta) = r_ij . r_ik / (r_ij r_ik), sin(theta) = sqrt(max(1 - cos^2, 0) + eps).
 * J layout: J[d * nnb * 3 + e * 3 + c] = dG[d] / d r_e[c]  (e = neighbour entry).
 */
void orc_center(const orc_desc* p, int nnb, const double* rv, const int32_t* sp,
                double* G, double* J)
{
    const int S = p->n_species, D = orc_descriptor_size(p);
    const int NR = p->n_rad, NT = p->n_theta, NA = p->n_ang_r;
    const double rc = p->rc;
    const double pref = pow(2.0, 1.0 - p->zeta);
    memset(G, 0, sizeof(double) * D);
    if (J) memset(J, 0, sizeof(double) * (size_t)D * nnb * 3);

    /* radial */
    for (int e = 0; e < nnb; ++e) {
        const double* r = rv + 3 * e;
        double rr = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        double fc = fcut(rr, rc), dfc = dfcut(rr, rc);
        for (int n = 0; n < NR; ++n) {
            double x = rr - p->rs_rad[n];
            double ga = exp(-p->eta_rad * x * x);
            int d = sp[e] * NR + n;
            G[d] += ga * fc;
            if (J) {
                double dv = ga * (-2.0 * p->eta_rad * x) * fc + ga * dfc; /* dG/dr */
                for (int c = 0; c < 3; ++c) J[(size_t)d * nnb * 3 + e * 3 + c] += dv * r[c] / rr;
            }
        }
    }

    if (p->angular_kind == 1) {
        /*
         * Standard BP angular term (Behler and Parrinello's G4, the form Sec. II.A cites next
         * to mBP), block of the unordered species pair {s_j, s_k}, index m*n_ang_r + n,
         * every unordered pair of distinct neighbour entries j < k counted once:
         *   G[...] += 2^(1-zeta_m) (1 + lambda_m cos(theta_ijk))^zeta_m   (0 where 1 + lambda cos <= 0)
         *             exp(-eta_n (r_ij^2 + r_ik^2 + r_jk^2)) f_c(r_ij) f_c(r_ik) f_c(r_jk)
         * with r_jk = |r_ik - r_ij| (the vectors of the two entries).
         */
        for (int e1 = 0; e1 < nnb; ++e1)
        for (int e2 = e1 + 1; e2 < nnb; ++e2) {
            const double* a = rv + 3 * e1; const double* b = rv + 3 * e2;
            double d[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
            double ra = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
            double rb = sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
            double rab = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            if (!(rab < rc)) continue;
            double cs = (a[0] * b[0] + a[1] * b[1] + a[2] * b[2]) / (ra * rb);
            double fa = fcut(ra, rc), fb = fcut(rb, rc), fab = fcut(rab, rc);
            double dfa = dfcut(ra, rc), dfb = dfcut(rb, rc), dfab = dfcut(rab, rc);
            double F3 = fa * fb * fab;
            double S2 = ra * ra + rb * rb + rab * rab;
            double dca[3], dcb[3], dF3a[3], dF3b[3], dSa[3], dSb[3];
            for (int c = 0; c < 3; ++c) {
                dca[c] = b[c] / (ra * rb) - cs * a[c] / (ra * ra);
                dcb[c] = a[c] / (ra * rb) - cs * b[c] / (rb * rb);
                /* d r_jk / d a = -(b - a)/r_jk, d r_jk / d b = (b - a)/r_jk */
                dF3a[c] = dfa * a[c] / ra * fb * fab - fa * fb * dfab * d[c] / rab;
                dF3b[c] = fa * dfb * b[c] / rb * fab + fa * fb * dfab * d[c] / rab;
                dSa[c] = 2.0 * a[c] - 2.0 * d[c];
                dSb[c] = 2.0 * b[c] + 2.0 * d[c];
            }
            int blk = S * NR + pair_block(sp[e1], sp[e2], S) * NT * NA;
            for (int m = 0; m < NT; ++m) {
                double lam = p->bp_lambda[m], zt = p->bp_zeta[m];
                double base = 1.0 + lam * cs;
                double A = 0.0, dA = 0.0;   /* A_m and dA_m / dcos */
                if (base > 0.0) {
                    A = pow(2.0, 1.0 - zt) * pow(base, zt);
                    dA = pow(2.0, 1.0 - zt) * zt * lam * pow(base, zt - 1.0);
                }
                for (int n = 0; n < NA; ++n) {
                    double B = exp(-p->bp_eta[n] * S2);
                    int dd = blk + m * NA + n;
                    G[dd] += A * B * F3;
                    if (J) {
                        for (int c = 0; c < 3; ++c) {
                            J[(size_t)dd * nnb * 3 + e1 * 3 + c] +=
                                dA * B * F3 * dca[c] - A * p->bp_eta[n] * B * F3 * dSa[c] + A * B * dF3a[c];
                            J[(size_t)dd * nnb * 3 + e2 * 3 + c] +=
                                dA * B * F3 * dcb[c] - A * p->bp_eta[n] * B * F3 * dSb[c] + A * B * dF3b[c];
                        }
                    }
                }
            }
        }
        return;
    }

    /* angular (mBP) */
    for (int e1 = 0; e1 < nnb; ++e1)
    for (int e2 = e1 + 1; e2 < nnb; ++e2) {
        const double* a = rv + 3 * e1; const double* b = rv + 3 * e2;
        double ra = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        double rb = sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
        double ab = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
        double cs = ab / (ra * rb);
        double one_m = 1.0 - cs * cs;
        double sn = sqrt((one_m > 0.0 ? one_m : 0.0) + p->eps_theta);
        double dsn_dcs = one_m > 0.0 ? -cs / sn : 0.0;
        double fa = fcut(ra, rc), fb = fcut(rb, rc), dfa = dfcut(ra, rc), dfb = dfcut(rb, rc);
        double rbar = 0.5 * (ra + rb);
        /* d cos / d a and d cos / d b */
        double dca[3], dcb[3];
        for (int c = 0; c < 3; ++c) {
            dca[c] = b[c] / (ra * rb) - cs * a[c] / (ra * ra);
            dcb[c] = a[c] / (ra * rb) - cs * b[c] / (rb * rb);
        }
        int blk = S * NR + pair_block(sp[e1], sp[e2], S) * NT * NA;
        for (int m = 0; m < NT; ++m) {
            double ct = cos(p->theta_s[m]), st = sin(p->theta_s[m]);
            double base = 1.0 + cs * ct + sn * st;
            double A = 0.0, dA = 0.0;  /* A_m and dA_m / dcos */
            if (base > 0.0) {
                A = pref * pow(base, p->zeta);
                dA = pref * p->zeta * pow(base, p->zeta - 1.0) * (ct + dsn_dcs * st);
            }
            for (int n = 0; n < NA; ++n) {
                double x = rbar - p->rs_ang[n];
                double ga = exp(-p->eta_ang * x * x);
                double B = ga * fa * fb;
                int d = blk + m * NA + n;
                G[d] += A * B;
                if (J) {
                    /* d B / d ra and d B / d rb (d rbar / d ra = 1/2) */
                    double dBa = ga * (-p->eta_ang * x) * fa * fb + ga * dfa * fb;
                    double dBb = ga * (-p->eta_ang * x) * fa * fb + ga * fa * dfb;
                    for (int c = 0; c < 3; ++c) {
                        J[(size_t)d * nnb * 3 + e1 * 3 + c] += dA * B * dca[c] + A * dBa * a[c] / ra;
                        J[(size_t)d * nnb * 3 + e2 * 3 + c] += dA * B * dcb[c] + A * dBb * b[c] / rb;
                    }
                }
            }
        }
    }
}

/* ------------------------------------------------------------------------- */
/* per-species MLP (Eq. 1)                                                    */
/* ------------------------------------------------------------------------- */

static double act_f(int t, double z)
{
    switch (t) {
    case 1: return exp(-z * z);
    case 2: return z > 0.0 ? z : 0.0;
    case 3: return tanh(z);
    default: return z;
    }
}
static double act_d1(int t, double z)
{
    switch (t) {
    case 1: return -2.0 * z * exp(-z * z);
    case 2: return z > 0.0 ? 1.0 : 0.0;
    case 3: { double th = tanh(z); return 1.0 - th * th; }
    default: return 1.0;
    }
}
static double act_d2(int t, double z)
{
    switch (t) {
    case 1: return (4.0 * z * z - 2.0) * exp(-z * z);
    case 3: { double th = tanh(z); return -2.0 * th * (1.0 - th * th); }
    default: return 0.0;
    }
}

int64_t orc_arch_nparams(const orc_arch* A)
{
    int64_t n = 0;
    for (int l = 0; l < A->n_layers; ++l) n += (int64_t)A->widths[l + 1] * A->widths[l] + A->widths[l + 1];
    return n;
}

static int max_width(const orc_arch* A)
{
    int w = 0;
    for (int l = 0; l <= A->n_layers; ++l) if (A->widths[l] > w) w = A->widths[l];
    return w;
}

/*
 * One atom through its species' network.  E = a^L (single output).  When g != NULL,
 * g = dE/dx by the chain rule.  When dtheta != NULL, accumulates
 *   d/dtheta [ alpha * E(x) + beta * (dE/dx(x) . xdot) ]
 * obtained by differentiating the forward pass and its tangent along xdot
 * (z_l = W_l a_{l-1} + b_l, zdot_l = W_l adot_{l-1}, adot_l = sigma'(z_l) zdot_l).
 */
void orc_mlp(const orc_arch* A, const double* th, const double* x, double* E, double* g,
             const double* xdot, double alpha, double beta, double* dtheta)
{
    const int L = A->n_layers, W = max_width(A);
    double* a = (double*)calloc((size_t)(L + 1) * W, sizeof(double));   /* a_l */
    double* z = (double*)calloc((size_t)(L + 1) * W, sizeof(double));   /* z_l */
    double* ad = (double*)calloc((size_t)(L + 1) * W, sizeof(double));  /* adot_l */
    double* zd = (double*)calloc((size_t)(L + 1) * W, sizeof(double));  /* zdot_l */
    double* bar = (double*)calloc(W, sizeof(double));
    double* bard = (double*)calloc(W, sizeof(double));
    double* nbar = (double*)calloc(W, sizeof(double));
    double* nbard = (double*)calloc(W, sizeof(double));
    const double** Wl = (const double**)calloc((size_t)(L > 0 ? L : 1), sizeof(double*));
    const double** bl = (const double**)calloc((size_t)(L > 0 ? L : 1), sizeof(double*));
    int64_t* offW = (int64_t*)calloc((size_t)(L > 0 ? L : 1), sizeof(int64_t));
    int64_t o = 0;
    for (int l = 0; l < L; ++l) {
        Wl[l] = th + o; offW[l] = o; o += (int64_t)A->widths[l + 1] * A->widths[l];
        bl[l] = th + o; o += A->widths[l + 1];
    }
    for (int k = 0; k < A->widths[0]; ++k) {
        a[k] = x[k];
        ad[k] = xdot ? xdot[k] : 0.0;
    }
    for (int l = 1; l <= L; ++l) {
        int ni = A->widths[l - 1], no = A->widths[l];
        for (int u = 0; u < no; ++u) {
            double s = bl[l - 1][u], sd = 0.0;
            for (int k = 0; k < ni; ++k) {
                s += Wl[l - 1][(size_t)u * ni + k] * a[(size_t)(l - 1) * W + k];
                sd += Wl[l - 1][(size_t)u * ni + k] * ad[(size_t)(l - 1) * W + k];
            }
            z[(size_t)l * W + u] = s;
            zd[(size_t)l * W + u] = sd;
            a[(size_t)l * W + u] = act_f(A->act[l - 1], s);
            ad[(size_t)l * W + u] = act_d1(A->act[l - 1], s) * sd;
        }
    }
    if (E) *E = a[(size_t)L * W + 0];

    if (g) {  /* plain backprop of E */
        bar[0] = 1.0;
        for (int l = L; l >= 1; --l) {
            int ni = A->widths[l - 1], no = A->widths[l];
            for (int k = 0; k < ni; ++k) nbar[k] = 0.0;
            for (int u = 0; u < no; ++u) {
                double zb = bar[u] * act_d1(A->act[l - 1], z[(size_t)l * W + u]);
                for (int k = 0; k < ni; ++k) nbar[k] += Wl[l - 1][(size_t)u * ni + k] * zb;
            }
            for (int k = 0; k < ni; ++k) bar[k] = nbar[k];
        }
        for (int k = 0; k < A->widths[0]; ++k) g[k] = bar[k];
    }

    if (dtheta) {  /* reverse pass over the forward + tangent computation */
        for (int k = 0; k < W; ++k) { bar[k] = 0.0; bard[k] = 0.0; }
        bar[0] = alpha;
        bard[0] = beta;
        for (int l = L; l >= 1; --l) {
            int ni = A->widths[l - 1], no = A->widths[l];
            int t = A->act[l - 1];
            for (int k = 0; k < ni; ++k) { nbar[k] = 0.0; nbard[k] = 0.0; }
            double* dW = dtheta + offW[l - 1];
            double* db = dW + (size_t)no * ni;
            for (int u = 0; u < no; ++u) {
                double zz = z[(size_t)l * W + u];
                double zb = bar[u] * act_d1(t, zz) + bard[u] * act_d2(t, zz) * zd[(size_t)l * W + u];
                double zdb = bard[u] * act_d1(t, zz);
                for (int k = 0; k < ni; ++k) {
                    dW[(size_t)u * ni + k] += zb * a[(size_t)(l - 1) * W + k] + zdb * ad[(size_t)(l - 1) * W + k];
                    nbar[k] += Wl[l - 1][(size_t)u * ni + k] * zb;
                    nbard[k] += Wl[l - 1][(size_t)u * ni + k] * zdb;
                }
                db[u] += zb;
            }
            for (int k = 0; k < ni; ++k) { bar[k] = nbar[k]; bard[k] = nbard[k]; }
        }
    }
    free(a); free(z); free(ad); free(zd); free(bar); free(bard); free(nbar); free(nbard);
    free(Wl); free(bl); free(offW);
}

/* ------------------------------------------------------------------------- */
/* whole batch                                                                */
/* ------------------------------------------------------------------------- */

/*
 * Neighbour list of every atom of a batch (atom_off[C+1]; positions, species, cells,
 * pbc as in the CUDA library).  Entries sorted by (i, j, n).  nbr_i/nbr_j are global
 * atom indices.  Returns the total count (entries beyond cap are counted, not written).
 */
int64_t orc_neighbor_list(int64_t n_cfg, const int64_t* atom_off, const double* pos,
                          const double* cell, const uint8_t* pbc, double rc, int64_t cap,
                          int64_t* nbr_i, int64_t* nbr_j, int32_t* shift)
{
    int64_t total = 0;
    orc_nb* buf = NULL;
    int64_t bcap = 0;
    for (int64_t c = 0; c < n_cfg; ++c) {
        int64_t a0 = atom_off[c], n = atom_off[c + 1] - a0;
        for (int64_t i = 0; i < n; ++i) {
            int64_t k = neighbours_of(i, n, pos + 3 * a0, NULL, cell + 9 * c, pbc + 3 * c, rc,
                                      NULL, 0, bcap, buf);
            if (k > bcap) {
                bcap = 2 * k + 16;
                buf = (orc_nb*)realloc(buf, sizeof(orc_nb) * bcap);
                k = neighbours_of(i, n, pos + 3 * a0, NULL, cell + 9 * c, pbc + 3 * c, rc,
                                  NULL, 0, bcap, buf);
            }
            qsort(buf, (size_t)k, sizeof(orc_nb), cmp_nb);
            for (int64_t e = 0; e < k; ++e, ++total) {
                if (total < cap) {
                    nbr_i[total] = a0 + i;
                    nbr_j[total] = a0 + buf[e].j;
                    for (int d = 0; d < 3; ++d) shift[3 * total + d] = buf[e].n[d];
                }
            }
        }
    }
    free(buf);
    return total;
}

/* neighbour entries of atom i (sorted), growing the buffer as needed */
static int64_t env(int64_t i, int64_t n, const double* pos, const int32_t* spec, const double* cell,
                   const uint8_t* pbc, double rc, const int64_t* cand, int64_t n_cand,
                   orc_nb** buf, int64_t* bcap)
{
    int64_t k = neighbours_of(i, n, pos, spec, cell, pbc, rc, cand, n_cand, *bcap, *buf);
    if (k > *bcap) {
        *bcap = 2 * k + 16;
        *buf = (orc_nb*)realloc(*buf, sizeof(orc_nb) * (*bcap));
        k = neighbours_of(i, n, pos, spec, cell, pbc, rc, cand, n_cand, *bcap, *buf);
    }
    qsort(*buf, (size_t)k, sizeof(orc_nb), cmp_nb);
    return k;
}

typedef struct {
    orc_nb* nb; int64_t cap;
    double* rv; int32_t* sp; int64_t rcap;
    double* G; double* J; double* g; double* w; double* v; int64_t jcap;
} orc_work;

static void work_fit(orc_work* wk, int64_t nnb, int D)
{
    if (nnb > wk->rcap) {
        wk->rcap = 2 * nnb + 16;
        wk->rv = (double*)realloc(wk->rv, sizeof(double) * 3 * wk->rcap);
        wk->sp = (int32_t*)realloc(wk->sp, sizeof(int32_t) * wk->rcap);
        wk->v = (double*)realloc(wk->v, sizeof(double) * 3 * wk->rcap);
    }
    int64_t need = (int64_t)D * (nnb > 0 ? nnb : 1) * 3;
    if (need > wk->jcap) {
        wk->jcap = 2 * need;
        wk->J = (double*)realloc(wk->J, sizeof(double) * wk->jcap);
    }
    if (!wk->G) {
        wk->G = (double*)calloc(D, sizeof(double));
        wk->g = (double*)calloc(D, sizeof(double));
        wk->w = (double*)calloc(D, sizeof(double));
    }
}

static void work_free(orc_work* wk)
{
    free(wk->nb); free(wk->rv); free(wk->sp); free(wk->G); free(wk->J); free(wk->g);
    free(wk->w); free(wk->v);
}

/*
 * Energies, forces, virials (and optionally descriptors, the loss and its parameter
 * gradient) of a batch.  theta holds all species' parameters; theta_off[s] is the
 * start of species s.  Outputs: G[N*D] (or NULL), E_atom[N], E_cfg[C], F[N*3],
 * virial[C*9] (or NULL).  Training (when E_ref != NULL):
 *   L = (1/C) sum_c (E_c - E_ref_c)^2 + w_force/(3N) sum_{m,a} (F_ma - F_ref_ma)^2
 * and dtheta (same layout as theta) = dL/dtheta, via
 *   alpha_c = 2/C (E_c - E_ref_c),  u = 2 w_force/(3N) (F - F_ref),
 *   w_i = sum_e dG_i/dr_e . (u_j(e) - u_i)   (descriptor JVP),
 *   dL/dtheta = sum_i d/dtheta [ alpha_c(i) E_i - g_i . w_i ].
 * Returns 0.
 */
/* Loss options of Sec. II.A: for the energy and the force terms a quadratic x^2 or an
 * exponential exp(x^2) - 1 function of the difference (the paper names both, without the
 * form; this reading equals the quadratic to leading order), energies per configuration or
 * per atom (difference divided by the configuration's atom count), and a penalty
 * l1 sum |w| + l2 sum w^2 over every weight (biases excluded). */
typedef struct { int32_t e_kind, f_kind, e_per_atom; double l1, l2; } orc_loss;

static double loss_term(int kind, double x) { return kind ? exp(x * x) - 1.0 : x * x; }
static double loss_slope(int kind, double x) { return kind ? 2.0 * x * exp(x * x) : 2.0 * x; }

int orc_batch(int64_t n_cfg, const int64_t* atom_off, const double* pos, const int32_t* species,
              const double* cell, const uint8_t* pbc, const orc_desc* p, const orc_arch* archs,
              const double* theta, const int64_t* theta_off,
              double* G_out, double* E_atom, double* E_cfg, double* F, double* virial,
              const double* E_ref, const double* F_ref, double w_force, double* loss, double* dtheta,
              const uint8_t* ghost, double c_norm, double n_norm, const orc_loss* lo)
{
    const orc_loss lq = {0, 0, 0, 0.0, 0.0};
    if (!lo) lo = &lq;
    const int D = orc_descriptor_size(p);
    const int64_t N = atom_off[n_cfg];
    /* Loss normalisers: the batch's own counts unless given (a shard of a larger batch). */
    const double CN = c_norm > 0.0 ? c_norm : (double)n_cfg;
    const double NN = n_norm > 0.0 ? n_norm : (double)N;
    orc_work wk;
    memset(&wk, 0, sizeof wk);
    work_fit(&wk, 16, D);
    memset(F, 0, sizeof(double) * 3 * N);
    if (virial) memset(virial, 0, sizeof(double) * 9 * n_cfg);

    for (int64_t c = 0; c < n_cfg; ++c) {
        int64_t a0 = atom_off[c], n = atom_off[c + 1] - a0;
        const double* cp = cell + 9 * c; const uint8_t* pp = pbc + 3 * c;
        double ec = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            /* The energy is a sum over centres (Sec. II); an atom flagged ghost is only a
             * neighbour, so the sum and its derivatives leave out its own term. */
            if (ghost && ghost[a0 + i]) {
                E_atom[a0 + i] = 0.0;
                if (G_out) memset(G_out + (size_t)(a0 + i) * D, 0, sizeof(double) * D);
                continue;
            }
            int64_t k = env(i, n, pos + 3 * a0, species + a0, cp, pp, p->rc, NULL, 0, &wk.nb, &wk.cap);
            work_fit(&wk, k, D);
            for (int64_t e = 0; e < k; ++e) {
                memcpy(wk.rv + 3 * e, wk.nb[e].r, sizeof(double) * 3);
                wk.sp[e] = wk.nb[e].sp;
            }
            orc_center(p, (int)k, wk.rv, wk.sp, wk.G, wk.J);
            int s = species[a0 + i];
            double Ei;
            orc_mlp(&archs[s], theta + theta_off[s], wk.G, &Ei, wk.g, NULL, 0.0, 0.0, NULL);
            if (G_out) memcpy(G_out + (size_t)(a0 + i) * D, wk.G, sizeof(double) * D);
            E_atom[a0 + i] = Ei;
            ec += Ei;
            /* q_e = J_e^T g ; F_i += q_e ; F_j -= q_e ; virial -= q (x) r */
            for (int64_t e = 0; e < k; ++e) {
                double q[3] = {0.0, 0.0, 0.0};
                for (int d = 0; d < D; ++d)
                    for (int cc = 0; cc < 3; ++cc) q[cc] += wk.J[(size_t)d * k * 3 + e * 3 + cc] * wk.g[d];
                int64_t j = a0 + wk.nb[e].j;
                for (int cc = 0; cc < 3; ++cc) {
                    F[3 * (a0 + i) + cc] += q[cc];
                    F[3 * j + cc] -= q[cc];
                }
                if (virial)
                    for (int aa = 0; aa < 3; ++aa)
                        for (int bb = 0; bb < 3; ++bb) virial[9 * c + 3 * aa + bb] -= q[aa] * wk.rv[3 * e + bb];
            }
        }
        E_cfg[c] = ec;
    }

    if (E_ref) {
        double le = 0.0, lf = 0.0, l1 = 0.0, l2 = 0.0;
        for (int64_t c = 0; c < n_cfg; ++c) {
            const int64_t n = atom_off[c + 1] - atom_off[c];
            double d = E_cfg[c] - E_ref[c];
            if (lo->e_per_atom && n > 0) d /= (double)n;
            le += loss_term(lo->e_kind, d);
        }
        for (int64_t t = 0; t < 3 * N; ++t) lf += loss_term(lo->f_kind, F[t] - F_ref[t]);
        const int S = p->n_species;
        for (int s = 0; s < S; ++s) {           /* weights of every layer, biases excluded */
            int64_t off = theta_off[s];
            for (int l = 0; l < archs[s].n_layers; ++l) {
                const int64_t nw = (int64_t)archs[s].widths[l + 1] * archs[s].widths[l];
                for (int64_t k = 0; k < nw; ++k) { l1 += fabs(theta[off + k]); l2 += theta[off + k] * theta[off + k]; }
                off += nw + archs[s].widths[l + 1];
            }
        }
        *loss = le / CN + w_force * lf / (3.0 * NN) + lo->l1 * l1 + lo->l2 * l2;
        if (dtheta) {
            memset(dtheta, 0, sizeof(double) * theta_off[S]);
            double* u = (double*)malloc(sizeof(double) * 3 * N);
            for (int64_t t = 0; t < 3 * N; ++t) u[t] = w_force / (3.0 * NN) * loss_slope(lo->f_kind, F[t] - F_ref[t]);
            for (int64_t c = 0; c < n_cfg; ++c) {
                int64_t a0 = atom_off[c], n = atom_off[c + 1] - a0;
                const double* cp = cell + 9 * c; const uint8_t* pp = pbc + 3 * c;
                const double per = (lo->e_per_atom && n > 0) ? 1.0 / (double)n : 1.0;
                double alpha = loss_slope(lo->e_kind, (E_cfg[c] - E_ref[c]) * per) * per / CN;
                for (int64_t i = 0; i < n; ++i) {
                    if (ghost && ghost[a0 + i]) continue;
                    int64_t k = env(i, n, pos + 3 * a0, species + a0, cp, pp, p->rc, NULL, 0, &wk.nb, &wk.cap);
                    work_fit(&wk, k, D);
                    for (int64_t e = 0; e < k; ++e) {
                        memcpy(wk.rv + 3 * e, wk.nb[e].r, sizeof(double) * 3);
                        wk.sp[e] = wk.nb[e].sp;
                        for (int cc = 0; cc < 3; ++cc)
                            wk.v[3 * e + cc] = u[3 * (a0 + wk.nb[e].j) + cc] - u[3 * (a0 + i) + cc];
                    }
                    orc_center(p, (int)k, wk.rv, wk.sp, wk.G, wk.J);
                    for (int d = 0; d < D; ++d) {
                        double s = 0.0;
                        for (int64_t e = 0; e < k; ++e)
                            for (int cc = 0; cc < 3; ++cc) s += wk.J[(size_t)d * k * 3 + e * 3 + cc] * wk.v[3 * e + cc];
                        wk.w[d] = s;
                    }
                    int s = species[a0 + i];
                    orc_mlp(&archs[s], theta + theta_off[s], wk.G, NULL, NULL, wk.w, alpha, -1.0,
                            dtheta + theta_off[s]);
                }
            }
            free(u);
            for (int s = 0; s < S; ++s) {       /* penalty gradient: l1 sign(w) + 2 l2 w */
                int64_t off = theta_off[s];
                for (int l = 0; l < archs[s].n_layers; ++l) {
                    const int64_t nw = (int64_t)archs[s].widths[l + 1] * archs[s].widths[l];
                    for (int64_t k = 0; k < nw; ++k) {
                        const double w = theta[off + k];
                        dtheta[off + k] += lo->l1 * ((w > 0.0) - (w < 0.0)) + 2.0 * lo->l2 * w;
                    }
                    off += nw + archs[s].widths[l + 1];
                }
            }
        }
    }
    work_free(&wk);
    return 0;
}

/* One Adam step (Kingma and Ba, Algorithm 1) for step t >= 1: m = b1 m + (1 - b1) g,
 * v = b2 v + (1 - b2) g^2, theta -= lr_t (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps),
 * with lr_t = lr0 rate^(t / steps) (exponential decay; steps = 0: constant).  Entries with
 * frozen[k] != 0 keep theta, m and v. */
void orc_adam_step(int64_t n, double* theta, const double* g, double* m, double* v, int64_t t, double lr0,
                   double rate, double steps, double b1, double b2, double eps, const uint8_t* frozen)
{
    const double lr = steps > 0.0 ? lr0 * pow(rate, (double)t / steps) : lr0;
    const double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
    for (int64_t k = 0; k < n; ++k) {
        if (frozen && frozen[k]) continue;
        m[k] = b1 * m[k] + (1.0 - b1) * g[k];
        v[k] = b2 * v[k] + (1.0 - b2) * g[k] * g[k];
        theta[k] -= lr * (m[k] / c1) / (sqrt(v[k] / c2) + eps);
    }
}

/*
 * Sampled evaluation inside one (possibly huge) configuration: for each sampled atom m,
 * its sorted neighbour list, descriptor, atomic energy and force.  The force needs the
 * networks of m's neighbours; every neighbour of a neighbour of m lies within 2 rc of
 * m, so all searches run over the atoms found within 2 rc of m (brute force over the
 * whole configuration once per sample).
 *   nb_j[ns*cap], nb_shift[ns*cap*3], nnb[ns] (count, may exceed cap), G[ns*D],
 *   E[ns], F[ns*3].
 */
int orc_sampled(int64_t n, const double* pos, const int32_t* species, const double* cell,
                const uint8_t* pbc, const orc_desc* p, const orc_arch* archs, const double* theta,
                const int64_t* theta_off, int64_t n_samples, const int64_t* samples, int64_t cap,
                int32_t* nb_j, int32_t* nb_shift, int64_t* nnb, double* G, double* E, double* F)
{
    const int D = orc_descriptor_size(p);
    orc_work wk;
    memset(&wk, 0, sizeof wk);
    work_fit(&wk, 16, D);
    orc_nb* far = NULL; int64_t fcap = 0;
    orc_nb* inner = NULL; int64_t icap = 0;
    int64_t* cand = NULL; int64_t ccap = 0;
    for (int64_t q = 0; q < n_samples; ++q) {
        int64_t m = samples[q];
        /* every atom with some image within 2 rc of m */
        int64_t kf = env(m, n, pos, species, cell, pbc, 2.0 * p->rc, NULL, 0, &far, &fcap);
        if (kf + 1 > ccap) { ccap = 2 * kf + 16; cand = (int64_t*)realloc(cand, sizeof(int64_t) * ccap); }
        int64_t nc = 0;
        cand[nc++] = m;
        for (int64_t e = 0; e < kf; ++e) {
            int64_t j = far[e].j;
            int seen = 0;
            for (int64_t t = 0; t < nc; ++t) if (cand[t] == j) { seen = 1; break; }
            if (!seen) cand[nc++] = j;
        }
        /* m itself */
        int64_t km = env(m, n, pos, species, cell, pbc, p->rc, cand, nc, &inner, &icap);
        nnb[q] = km;
        for (int64_t e = 0; e < km && e < cap; ++e) {
            nb_j[q * cap + e] = inner[e].j;
            for (int d = 0; d < 3; ++d) nb_shift[(q * cap + e) * 3 + d] = inner[e].n[d];
        }
        work_fit(&wk, km, D);
        for (int64_t e = 0; e < km; ++e) { memcpy(wk.rv + 3 * e, inner[e].r, 24); wk.sp[e] = inner[e].sp; }
        orc_center(p, (int)km, wk.rv, wk.sp, wk.G, wk.J);
        int s = species[m];
        orc_mlp(&archs[s], theta + theta_off[s], wk.G, &E[q], wk.g, NULL, 0.0, 0.0, NULL);
        memcpy(G + (size_t)q * D, wk.G, sizeof(double) * D);
        double f[3] = {0.0, 0.0, 0.0};
        for (int64_t e = 0; e < km; ++e)
            for (int d = 0; d < D; ++d)
                for (int cc = 0; cc < 3; ++cc) f[cc] += wk.J[(size_t)d * km * 3 + e * 3 + cc] * wk.g[d];
        /* distinct neighbour atoms a of m: subtract their q entries that point at m */
        int64_t* atoms = (int64_t*)malloc(sizeof(int64_t) * (km + 1));
        int64_t na = 0;
        for (int64_t e = 0; e < km; ++e) {
            int64_t a = inner[e].j;
            int seen = 0;
            for (int64_t t = 0; t < na; ++t) if (atoms[t] == a) { seen = 1; break; }
            if (!seen) atoms[na++] = a;
        }
        for (int64_t t = 0; t < na; ++t) {
            int64_t a = atoms[t];
            orc_nb* nba = NULL; int64_t bc = 0;
            int64_t ka = env(a, n, pos, species, cell, pbc, p->rc, cand, nc, &nba, &bc);
            work_fit(&wk, ka, D);
            for (int64_t e = 0; e < ka; ++e) { memcpy(wk.rv + 3 * e, nba[e].r, 24); wk.sp[e] = nba[e].sp; }
            orc_center(p, (int)ka, wk.rv, wk.sp, wk.G, wk.J);
            int sa = species[a];
            orc_mlp(&archs[sa], theta + theta_off[sa], wk.G, NULL, wk.g, NULL, 0.0, 0.0, NULL);
            for (int64_t e = 0; e < ka; ++e) {
                if (nba[e].j != m) continue;
                for (int d = 0; d < D; ++d)
                    for (int cc = 0; cc < 3; ++cc) f[cc] -= wk.J[(size_t)d * ka * 3 + e * 3 + cc] * wk.g[d];
            }
            free(nba);
        }
        free(atoms);
        for (int cc = 0; cc < 3; ++cc) F[3 * q + cc] = f[cc];
    }
    free(far); free(inner); free(cand);
    work_free(&wk);
    return 0;
}

/* ------------------------------------------------------------------ Langevin dynamics
 *
 * Units: positions A, velocities A/fs, time fs, masses amu, energies eV, temperature K.
 * Acceleration of a force of 1 eV/A on 1 amu: e / (amu 1e-10 m) = 9.648533212e17 m/s^2
 * = 9.648533212e-3 A/fs^2.  Boltzmann constant 8.617333262e-5 eV/K (exact SI values).
 */
#define ORC_ACC 9.648533212e-3
#define ORC_KB 8.617333262e-5

/* Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1,
 * 2, 3", SC'11): ten rounds on a counter of four 32-bit words with a key of two; each round
 * multiplies words 0 and 2 by two constants (64-bit products split in high and low halves),
 * mixes the high halves with the other words and the key, and the key advances by two Weyl
 * constants between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3], k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        const uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Three standard normal numbers for atom a at step t: the four words of Philox with
 * counter (a low, a high, t low, t high) and key (seed low, seed high), as uniforms
 * u = (x + 1/2) 2^-32 in (0, 1), through Box-Muller: sqrt(-2 ln u0) (cos, sin)(2 pi u1),
 * sqrt(-2 ln u2) cos(2 pi u3). */
void orc_gauss3(uint64_t seed, int64_t a, int64_t t, double g[3])
{
    const uint32_t ctr[4] = {(uint32_t)a, (uint32_t)((uint64_t)a >> 32), (uint32_t)t, (uint32_t)((uint64_t)t >> 32)};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    double u[4];
    for (int k = 0; k < 4; ++k) u[k] = ((double)x[k] + 0.5) * (1.0 / 4294967296.0);
    const double two_pi = 6.283185307179586476925286766559;
    const double r01 = sqrt(-2.0 * log(u[0])), r23 = sqrt(-2.0 * log(u[2]));
    g[0] = r01 * cos(two_pi * u[1]);
    g[1] = r01 * sin(two_pi * u[1]);
    g[2] = r23 * cos(two_pi * u[3]);
}

/* BAOAB Langevin dynamics (Leimkuhler and Matthews, 2013) on every configuration of a
 * batch, forces from orc_batch at every step (no neighbour-list reuse):
 *   B: v += dt/2 F/m;  A: x += dt/2 v;  O: v = c1 v + c2 sqrt(kB T / m) g;  A: x += dt/2 v;
 *   F = F(x);  B: v += dt/2 F/m;     c1 = exp(-friction dt), c2 = sqrt(1 - c1^2),
 * g the three normals of orc_gauss3(seed, atom, step0 + step).  With temperature 0 and
 * friction 0 this is velocity Verlet.  pos, vel [N*3] in/out; F [N*3] out (forces at the
 * final positions); E_traj [n_steps * n_cfg] (may be NULL): energies after each step. */
int orc_md_baoab(int64_t n_cfg, const int64_t* atom_off, double* pos, double* vel, const int32_t* species,
                 const double* cell, const uint8_t* pbc, const orc_desc* p, const orc_arch* archs,
                 const double* theta, const int64_t* theta_off, const double* mass, double dt,
                 double temperature, double friction, uint64_t seed, int64_t step0, int64_t n_steps,
                 double* F, double* E_traj)
{
    const int64_t N = atom_off[n_cfg];
    double* E_atom = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    double* E_cfg = (double*)malloc(sizeof(double) * (size_t)n_cfg);
    orc_batch(n_cfg, atom_off, pos, species, cell, pbc, p, archs, theta, theta_off, NULL, E_atom, E_cfg, F, NULL,
              NULL, NULL, 0.0, NULL, NULL, NULL, 0.0, 0.0, NULL);
    const double c1 = exp(-friction * dt), c2 = sqrt(1.0 - c1 * c1);
    const int thermostat = friction > 0.0 || temperature > 0.0;
    for (int64_t t = 0; t < n_steps; ++t) {
        for (int64_t i = 0; i < N; ++i) {
            const double a = ORC_ACC / mass[species[i]];
            double g[3] = {0.0, 0.0, 0.0};
            if (thermostat) orc_gauss3(seed, i, step0 + t, g);
            const double sig = sqrt(ORC_KB * temperature * a);
            for (int d = 0; d < 3; ++d) {
                double v = vel[3 * i + d] + 0.5 * dt * F[3 * i + d] * a;
                double x = pos[3 * i + d] + 0.5 * dt * v;
                if (thermostat) v = c1 * v + c2 * sig * g[d];
                x += 0.5 * dt * v;
                vel[3 * i + d] = v;
                pos[3 * i + d] = x;
            }
        }
        orc_batch(n_cfg, atom_off, pos, species, cell, pbc, p, archs, theta, theta_off, NULL, E_atom, E_cfg, F,
                  NULL, NULL, NULL, 0.0, NULL, NULL, NULL, 0.0, 0.0, NULL);
        for (int64_t i = 0; i < N; ++i) {
            const double a = ORC_ACC / mass[species[i]];
            for (int d = 0; d < 3; ++d) vel[3 * i + d] += 0.5 * dt * F[3 * i + d] * a;
        }
        if (E_traj) memcpy(E_traj + t * n_cfg, E_cfg, sizeof(double) * (size_t)n_cfg);
    }
    free(E_atom);
    free(E_cfg);
    return 0;
}
