// Langevin dynamics on the device (BAOAB splitting, Leimkuhler and Matthews): every
// configuration of a batch advances its own trajectory; the potential is the PANNA
// energy/force path of the rest of the library (Sec. II), evaluated once per step.  The
// paper times Langevin MD on a small carbon cell (Sec. III.B); it does not name the
// integrator.
//
// Units: positions A, velocities A/fs, time fs, masses amu, energies eV, temperature K.
// The noise is Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC'11) with counter
// (atom, step) and key seed, turned into normals by Box-Muller, so a trajectory does not
// depend on the launch shape.
#include "common.cuh"

namespace panna {

// Philox4x32-10: ten rounds of two 32 x 32 -> 64-bit products on words 0 and 2 of the
// counter, the high halves mixed with words 1, 3 and the key, the key advanced by two Weyl
// constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k.x += W0; k.y += W1; }
        const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// three standard normals of atom a at step t (Box-Muller on u = (x + 1/2) 2^-32)
__device__ __forceinline__ void gauss3(uint64_t seed, int64_t a, int64_t t, double g[3])
{
    const uint4 x = philox4x32_10(make_uint4((uint32_t)a, (uint32_t)((uint64_t)a >> 32), (uint32_t)t,
                                             (uint32_t)((uint64_t)t >> 32)),
                                  make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    const double s32 = 1.0 / 4294967296.0;
    const double u0 = ((double)x.x + 0.5) * s32, u1 = ((double)x.y + 0.5) * s32;
    const double u2 = ((double)x.z + 0.5) * s32, u3 = ((double)x.w + 0.5) * s32;
    const double r01 = sqrt(-2.0 * log(u0)), r23 = sqrt(-2.0 * log(u2));
    double s1, c1, s3, c3;
    sincospi(2.0 * u1, &s1, &c1);
    sincospi(2.0 * u3, &s3, &c3);
    g[0] = r01 * c1;
    g[1] = r01 * s1;
    g[2] = r23 * c3;
}

// B A O A: v += dt/2 a F; x += dt/2 v; v = c1 v + c2 sigma g; x += dt/2 v.  With a
// reference (positions of the last neighbour build), an atom that has moved more than
// sqrt(lim2) since then raises *stale.
__global__ void k_md_baoa(int64_t N, const int32_t* __restrict__ species, MdSpecies ms, double* __restrict__ pos,
                          double* __restrict__ vel, const float* __restrict__ F, double dt, double c1, double c2,
                          int thermostat, uint64_t seed, int64_t step, const double* __restrict__ pos_ref,
                          double lim2, int32_t* __restrict__ stale)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int sp = species[i];
    const double a = ms.acc[sp], sig = ms.sigma[sp];
    double g[3] = {0.0, 0.0, 0.0};
    if (thermostat) gauss3(seed, i, step, g);
    double d2 = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double v = vel[3 * i + d] + 0.5 * dt * (double)F[3 * i + d] * a;
        double x = pos[3 * i + d] + 0.5 * dt * v;
        if (thermostat) v = c1 * v + c2 * sig * g[d];
        x += 0.5 * dt * v;
        vel[3 * i + d] = v;
        pos[3 * i + d] = x;
        if (pos_ref) { const double e = x - pos_ref[3 * i + d]; d2 += e * e; }
    }
    if (pos_ref && d2 > lim2) *stale = 1;
}

// B: v += dt/2 a F
__global__ void k_md_b(int64_t N, const int32_t* __restrict__ species, MdSpecies ms, double* __restrict__ vel,
                       const float* __restrict__ F, double dt)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double a = ms.acc[species[i]];
#pragma unroll
    for (int d = 0; d < 3; ++d) vel[3 * i + d] += 0.5 * dt * (double)F[3 * i + d] * a;
}

cudaError_t launch_md_baoa(int64_t N, const int32_t* species, const MdSpecies& ms, double* pos, double* vel,
                           const float* F, double dt, double c1, double c2, int thermostat, uint64_t seed,
                           int64_t step, const double* pos_ref, double lim2, int32_t* stale, cudaStream_t s)
{
    if (N == 0) return cudaSuccess;
    k_md_baoa<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, species, ms, pos, vel, F, dt, c1, c2, thermostat, seed,
                                                          step, pos_ref, lim2, stale);
    return cudaGetLastError();
}

cudaError_t launch_md_b(int64_t N, const int32_t* species, const MdSpecies& ms, double* vel, const float* F,
                        double dt, cudaStream_t s)
{
    if (N == 0) return cudaSuccess;
    k_md_b<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, species, ms, vel, F, dt);
    return cudaGetLastError();
}

}  // namespace panna
