// Charge equilibration (Sec. II.B): every atom's network gives three outputs, the local
// energy e_i and corrections to the electronegativity and hardness of its species,
// chi_i = chi0_s + out_1, J_i = J0_s + out_2.  The charges of a configuration are the
// stationary point of
//     E(q) = sum_i (e_i + chi_i q_i + J_i q_i^2 / 2) + 1/2 sum_ij q_i q_j K_ij
// under sum_i q_i = Q_c, with Gaussian charges of per-species width sigma:
//     K_ij = ke erf(r_ij / g_ij) / r_ij,  g_ij = sqrt(2 (sigma_i^2 + sigma_j^2)),
//     K_ii = ke / (sigma_i sqrt(pi)),
// i.e. the linear system [A 1; 1^T 0] [q; lam] = [-chi; Q_c], A = diag(J) + K.
//
// k_qeq: one CTA per configuration (up to kQeqMax atoms, no periodic direction), launched
// once per size class (up to 32 atoms with 11 kB of shared memory, up to kQeqMax with
// 142 kB) so that small clusters keep many CTAs per SM and no host read sizes it.  The
// (n+1)^2 system is built in shared memory and solved in FP64 by Gaussian elimination with
// partial pivoting (the saddle-point matrix has a zero diagonal entry); then per atom the
// energy share e_i + chi_i q_i + J_i q_i^2/2 + q_i (K q)_i / 2, the Gaussian-charge pair
// forces, and the seeds (1, q_i, q_i^2/2) of the networks' input gradient.  The forces need
// no derivative of the charges: dE/dq is the multiplier times a constant vector, whose
// product with dq vanishes on the constraint.
#include <math.h>

#include "common.cuh"

namespace panna {

constexpr int kQeqThreads = 128;

// Gaussian-charge pair interaction and its derivative with respect to r, in single
// precision (relative error ~1e-7, far inside the FP32 force tolerance; the matrix, the
// solve and every sum stay FP64): FP64 square roots, divisions and transcendentals on the
// GB300's narrow FP64 pipe made this the slowest part of the call.
__device__ __forceinline__ void qeq_pair(float r, float si, float sj, float ke, float& K, float& dK)
{
    const float ig = rsqrtf(2.f * (si * si + sj * sj));
    const float t = r * ig;
    const float e = erff(t);
    const float ir = 1.f / r;
    K = ke * e * ir;
    dK = ke * ir * (1.1283791670955126f * __expf(-t * t) * ig - e * ir);
}

// distance of two staged atoms (FP64 positions, difference rounded to FP32)
__device__ __forceinline__ float qeq_dist(const double* px, const double* py, const double* pz, int i, int j,
                                          float& dx, float& dy, float& dz)
{
    dx = (float)(px[i] - px[j]);
    dy = (float)(py[i] - py[j]);
    dz = (float)(pz[i] - pz[j]);
    return sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
}

// Shared-memory workspace of one configuration (n atoms, n1 = n + 1 unknowns): the FP64
// matrix (kept for residuals), its FP32 LU factors, the permutation, right-hand side,
// solution, residual and correction, and the per-atom staging arrays.
struct QeqShared {
    double* M; float* LU; int* perm; double* rhs; double* x; double* res; float* d;
    double* px; double* py; double* pz; double* sg; double* chi; double* hd; double* ee;
};

__host__ __device__ inline size_t qeq_shared_bytes(int n)
{
    const size_t n1 = (size_t)n + 1;
    const size_t dbl = n1 * n1 + 3 * n1 + 7 * (size_t)n;   // M, rhs, x, res, staging
    const size_t flt = n1 * n1 + n1;                       // LU, d
    return dbl * sizeof(double) + ((flt * sizeof(float) + n1 * sizeof(int) + 7) & ~(size_t)7);
}

__device__ inline QeqShared qeq_carve(double* base, int n)
{
    const int n1 = n + 1;
    QeqShared q;
    q.M = base;
    q.rhs = q.M + n1 * n1; q.x = q.rhs + n1; q.res = q.x + n1;
    q.px = q.res + n1; q.py = q.px + n; q.pz = q.py + n;
    q.sg = q.pz + n; q.chi = q.sg + n; q.hd = q.chi + n; q.ee = q.hd + n;
    q.LU = reinterpret_cast<float*>(q.ee + n);
    q.d = q.LU + n1 * n1;
    q.perm = reinterpret_cast<int*>(q.d + n1);
    return q;
}

// x = LU^-1 P r in FP32 (one warp): forward substitution with the unit lower factor, then
// back substitution with the upper one; d holds the result
__device__ void qeq_lu_apply(const QeqShared& q, int n1, const double* r, int tid)
{
    if (tid >= 32) return;
    for (int k = 0; k < n1; ++k) {
        float acc = 0.f;
        for (int j = tid; j < k; j += 32) acc += q.LU[k * n1 + j] * q.d[j];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (tid == 0) q.d[k] = (float)r[q.perm[k]] - acc;
        __syncwarp();
    }
    for (int k = n1 - 1; k >= 0; --k) {
        float acc = 0.f;
        for (int j = k + 1 + tid; j < n1; j += 32) acc += q.LU[k * n1 + j] * q.d[j];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (tid == 0) q.d[k] = (q.d[k] - acc) / q.LU[k * n1 + k];
        __syncwarp();
    }
}

// Solves [A 1; 1^T 0] x = rhs (q.M, q.rhs) into q.x: LU factors with partial pivoting in FP32,
// then iterative refinement with FP64 residuals r = rhs - M x (two steps take the FP32
// solution to about FP64 accuracy for these well-conditioned systems; the FP64 work is
// O(n^2) instead of the O(n^3) of an FP64 factorisation, which the GB300's narrow FP64 pipe
// made the slowest part of the call).  Returns false (the same on every thread) for a zero
// or non-finite pivot.
__device__ bool qeq_solve(const QeqShared& q, int n1, int tid, int nt, int& piv, int& bad)
{
    for (int idx = tid; idx < n1 * n1; idx += nt) q.LU[idx] = (float)q.M[idx];
    for (int i = tid; i < n1; i += nt) q.perm[i] = i;
    __syncthreads();
    for (int k = 0; k < n1; ++k) {
        if (tid < 32) {
            float best = -1.f;
            int bi = k;
            for (int i = k + tid; i < n1; i += 32) {
                const float a = fabsf(q.LU[i * n1 + k]);
                if (a > best) { best = a; bi = i; }
            }
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
                const float ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (tid == 0) {
                piv = bi;
                if (!(best > 0.f) || !isfinite(best)) bad = 1;
            }
        }
        __syncthreads();
        if (bad) return false;
        const int p = piv;
        if (p != k) {
            for (int j = tid; j < n1; j += nt) {
                const float t = q.LU[k * n1 + j];
                q.LU[k * n1 + j] = q.LU[p * n1 + j];
                q.LU[p * n1 + j] = t;
            }
            if (tid == 0) {
                const int t = q.perm[k];
                q.perm[k] = q.perm[p];
                q.perm[p] = t;
            }
        }
        __syncthreads();
        const float inv = 1.f / q.LU[k * n1 + k];
        for (int i = k + 1 + tid; i < n1; i += nt) q.LU[i * n1 + k] *= inv;   // multipliers
        __syncthreads();
        const int m = n1 - k - 1;
        for (int idx = tid; idx < m * m; idx += nt) {
            const int i = k + 1 + idx / m, j = k + 1 + (idx - (idx / m) * m);
            q.LU[i * n1 + j] -= q.LU[i * n1 + k] * q.LU[k * n1 + j];
        }
        __syncthreads();
    }
    // solution and two refinement steps
    for (int i = tid; i < n1; i += nt) { q.x[i] = 0.0; q.res[i] = q.rhs[i]; }
    __syncthreads();
    for (int it = 0; it < 3; ++it) {
        qeq_lu_apply(q, n1, q.res, tid);
        __syncthreads();
        for (int i = tid; i < n1; i += nt) q.x[i] += (double)q.d[i];
        __syncthreads();
        if (it == 2) break;
        for (int i = tid; i < n1; i += nt) {
            double r = q.rhs[i];
            for (int j = 0; j < n1; ++j) r -= q.M[i * n1 + j] * q.x[j];
            q.res[i] = r;
        }
        __syncthreads();
    }
    return true;
}

// TRAIN = false: the charges, energies, pair forces and input-gradient seeds of the forward
// pass.  TRAIN = true: the charges' response for the loss gradient.  With u = dL/dF, the
// output tangents odot of the networks along the descriptor tangent of u, and the charge
// term's slope,
//   h_i = -(odot_i,1 + q_i odot_i,2 + sum_j q_j K'_ij (x_i - x_j).(u_i - u_j) / r_ij)
//         + 2 w_q (q_i - q_ref_i),
// the same matrix gives [A 1; 1^T 0][mu; nu] = [h; 0]; the reverse pass of the networks then
// takes the seeds (alpha_c, alpha_c q_i - mu_i, alpha_c q_i^2/2 - mu_i q_i) on the outputs and
// (-1, -q_i, -q_i^2/2) on their tangents.
template <bool TRAIN>
__global__ void __launch_bounds__(kQeqThreads)
k_qeq(QeqDev qp, panna_system sys, int64_t C, const int32_t* __restrict__ row_of_atom, const float* __restrict__ out,
      int ldo, const double* __restrict__ Qtot, float* __restrict__ E_rows, double* __restrict__ charges,
      float* __restrict__ F, float* __restrict__ seeds, int lds, DevStatus* status, int n_lo, int n_hi, QeqTrain tr)
{
    extern __shared__ double sm[];
    __shared__ int piv, bad;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int64_t c = blockIdx.x; c < C; c += gridDim.x) {
        const int64_t a0 = sys.atom_off[c];
        const int64_t n64 = sys.atom_off[c + 1] - a0;
        if (n64 <= n_lo || (n64 > n_hi && n_hi < kQeqMax)) continue;   // another size class
        const int n = (int)(n64 > kQeqMax ? kQeqMax + 1 : n64);
        if (n > kQeqMax || sys.pbc[3 * c] || sys.pbc[3 * c + 1] || sys.pbc[3 * c + 2]) {
            if (tid == 0) set_status(status, PANNA_ERR_UNSUPPORTED, (int)c);
            continue;
        }
        __syncthreads();   // the previous configuration's shared data is no longer read
        const int n1 = n + 1;
        const QeqShared qs = qeq_carve(sm, n);
        double* M = qs.M; double* rhs = qs.rhs; double* x = qs.x;
        double* px = qs.px; double* py = qs.py; double* pz = qs.pz;
        double* sg = qs.sg; double* chi = qs.chi; double* hd = qs.hd; double* ee = qs.ee;
        for (int i = tid; i < n; i += nt) {
            const int64_t a = a0 + i;
            const int64_t r = row_of_atom[a];
            const int s = sys.species[a];
            px[i] = sys.pos[3 * a]; py[i] = sys.pos[3 * a + 1]; pz[i] = sys.pos[3 * a + 2];
            sg[i] = qp.sigma[s];
            chi[i] = qp.chi0[s] + out[r * ldo + 1];
            hd[i] = qp.hard0[s] + out[r * ldo + 2];
            // forward: the local energy; response: the charge of the forward pass
            ee[i] = TRAIN ? tr.q[a] : out[r * ldo];
        }
        if (tid == 0) bad = 0;
        __syncthreads();
        const double self = qp.ke / sqrt(M_PI);
        // upper triangle and diagonal computed, mirrored below the diagonal
        for (int idx = tid; idx < n1 * n1; idx += nt) {
            const int i = idx / n1, j = idx - (idx / n1) * n1;
            if (j < i) continue;
            double v;
            if (j < n) {
                if (i == j) {
                    v = hd[i] + self / sg[i];
                } else {
                    float dx, dy, dz, K, dK;
                    qeq_pair(qeq_dist(px, py, pz, i, j, dx, dy, dz), (float)sg[i], (float)sg[j], (float)qp.ke, K, dK);
                    v = K;
                }
            } else {
                v = i == n ? 0.0 : 1.0;
            }
            M[idx] = v;
            M[j * n1 + i] = v;
        }
        if (!TRAIN) {
            for (int i = tid; i < n1; i += nt) rhs[i] = i < n ? -chi[i] : (Qtot ? Qtot[c] : 0.0);
        } else {
            for (int i = tid; i < n1; i += nt) {
                if (i == n) {
                    rhs[i] = 0.0;
                    continue;
                }
                const int64_t a = a0 + i;
                const int64_t r = row_of_atom[a];
                const double qi = ee[i];
                const float ux = tr.u[3 * a], uy = tr.u[3 * a + 1], uz = tr.u[3 * a + 2];
                double v = tr.odot[r * ldo + 1] + qi * tr.odot[r * ldo + 2];
                for (int j = 0; j < n; ++j) {
                    if (j == i) continue;
                    float dx, dy, dz, K, dK;
                    const float rr = qeq_dist(px, py, pz, i, j, dx, dy, dz);
                    qeq_pair(rr, (float)sg[i], (float)sg[j], (float)qp.ke, K, dK);
                    const int64_t b = a0 + j;
                    const float du = dx * (ux - tr.u[3 * b]) + dy * (uy - tr.u[3 * b + 1]) + dz * (uz - tr.u[3 * b + 2]);
                    v += ee[j] * (double)(dK * du / rr);
                }
                double h = -v;
                if (tr.q_ref) h += 2.0 * tr.w_charge * (qi - tr.q_ref[a]);
                rhs[i] = h;
            }
        }
        __syncthreads();
        if (!qeq_solve(qs, n1, tid, nt, piv, bad)) {
            if (tid == 0) set_status(status, PANNA_ERR_BAD_INPUT, (int)c);
            continue;
        }

        if (TRAIN) {
            const double al = tr.alpha[c];
            double lq = 0.0;
            for (int i = tid; i < n; i += nt) {
                const int64_t a = a0 + i;
                const int64_t r = row_of_atom[a];
                const double qi = ee[i], mu = x[i];
                seeds[r * lds] = (float)al;
                seeds[r * lds + 1] = (float)(al * qi - mu);
                seeds[r * lds + 2] = (float)(al * 0.5 * qi * qi - mu * qi);
                tr.seeds_t[r * lds] = -1.f;
                tr.seeds_t[r * lds + 1] = (float)(-qi);
                tr.seeds_t[r * lds + 2] = (float)(-0.5 * qi * qi);
                if (tr.q_ref) lq += tr.w_charge * (qi - tr.q_ref[a]) * (qi - tr.q_ref[a]);
            }
            if (tr.q_ref) {
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) lq += __shfl_xor_sync(0xffffffffu, lq, o);
                if ((tid & 31) == 0 && lq != 0.0) atomicAdd(tr.loss, lq);
            }
            continue;
        }
        // energies, pair forces, network seeds
        for (int i = tid; i < n; i += nt) {
            // sums of O(n) single-precision terms (FP32 accuracy is what the outputs carry)
            const double qi = x[i];
            const float qf = (float)qi;
            float kq = (float)(self / sg[i]) * qf, fx = 0.f, fy = 0.f, fz = 0.f;
            const float si = (float)sg[i], ke = (float)qp.ke;
            for (int j = 0; j < n; ++j) {
                if (j == i) continue;
                float dx, dy, dz, K, dK;
                const float r = qeq_dist(px, py, pz, i, j, dx, dy, dz);
                qeq_pair(r, si, (float)sg[j], ke, K, dK);
                const float xj = (float)x[j];
                kq = fmaf(K, xj, kq);
                const float f = -qf * xj * (dK / r);
                fx = fmaf(f, dx, fx); fy = fmaf(f, dy, fy); fz = fmaf(f, dz, fz);
            }
            const int64_t a = a0 + i;
            const int64_t r = row_of_atom[a];
            E_rows[r] = (float)(ee[i] + chi[i] * qi + 0.5 * hd[i] * qi * qi + 0.5 * qi * (double)kq);
            if (charges) charges[a] = qi;
            F[3 * a] += fx;
            F[3 * a + 1] += fy;
            F[3 * a + 2] += fz;
            seeds[r * lds] = 1.f;
            seeds[r * lds + 1] = (float)qi;
            seeds[r * lds + 2] = (float)(0.5 * qi * qi);
        }
    }
}

size_t qeq_smem_bytes(int max_n) { return qeq_shared_bytes(max_n); }

template <bool TRAIN>
static cudaError_t qeq_launch(const QeqDev& qp, const Work& w, const float* out, int ldo, const double* Qtot,
                              float* E_rows, double* charges, float* F, float* seeds, int lds, const QeqTrain& tr,
                              cudaStream_t s, int* launches)
{
    if (w.C == 0) return cudaSuccess;
    const int classes[3] = {0, 32, kQeqMax};
    cudaError_t e = cudaFuncSetAttribute(k_qeq<TRAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)qeq_smem_bytes(kQeqMax));
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (int k = 0; k < 2; ++k) {
        // resident CTAs of the class, each looping over the configurations; the last class
        // also reports configurations beyond kQeqMax
        const size_t smem = qeq_smem_bytes(classes[k + 1]);
        int per = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_qeq<TRAIN>, kQeqThreads, smem);
        int64_t nb = (int64_t)(sms > 0 ? sms : 1) * (per > 0 ? per : 1);
        if (nb > w.C) nb = w.C;
        k_qeq<TRAIN><<<(unsigned)nb, kQeqThreads, smem, s>>>(qp, *w.sys, w.C, w.row_of_atom, out, ldo, Qtot, E_rows,
                                                             charges, F, seeds, lds, w.status, classes[k],
                                                             classes[k + 1], tr);
        ++*launches;
    }
    return cudaGetLastError();
}

cudaError_t launch_qeq(const QeqDev& qp, const Work& w, const float* out, int ldo, const double* Qtot,
                       float* E_rows, double* charges, float* F, float* seeds, int lds, cudaStream_t s,
                       int* launches)
{
    return qeq_launch<false>(qp, w, out, ldo, Qtot, E_rows, charges, F, seeds, lds, QeqTrain{}, s, launches);
}

cudaError_t launch_qeq_response(const QeqDev& qp, const Work& w, const float* out, int ldo, const QeqTrain& tr,
                                float* seeds, int lds, cudaStream_t s, int* launches)
{
    return qeq_launch<true>(qp, w, out, ldo, nullptr, nullptr, nullptr, nullptr, seeds, lds, tr, s, launches);
}

}  // namespace panna
