// Internal interface of the per-species network kernels.
#pragma once

#include "common.cuh"

namespace panna {

constexpr int kBM = 64, kBN = 64, kBK = 16;      // weight-gradient tiles (k_wgrad)
constexpr int kGM = 128, kGN = 128, kGK = 8;     // layer GEMM tiles (k_gemm): 256 threads, 8 x 8 outputs each
enum { PRO_NONE = 0, PRO_DACT = 1 };
enum { EPI_STORE = 0, EPI_FWD = 1, EPI_TAN = 2 };

// Per-species shape of one layer as a kernel argument.
struct LayerArgs {
    int S;
    int K[kMaxSpecies], N[kMaxSpecies], act[kMaxSpecies], pact[kMaxSpecies];
    int64_t w_off[kMaxSpecies], b_off[kMaxSpecies];
};

// Host-side description of all species' networks (same depth for every species).
struct MlpPlan {
    int S, L;
    int widths[kMaxSpecies][kMaxLayers + 1];
    int acts[kMaxSpecies][kMaxLayers];
    int64_t w_off[kMaxSpecies][kMaxLayers], b_off[kMaxSpecies][kMaxLayers];
    int ld[kMaxLayers + 1];   // row stride of layer-l activations = max width over species
    int64_t P;                // total parameters
    int max_hidden;           // max over l >= 1 of ld[l]
    int n_out;                // output width: 1 (energy) or 3 (charge equilibration)
};

// Device buffers of one evaluation (rows in species order).
struct MlpBuffers {
    const float* G;                 // [N, ld[0]]
    float* Z[kMaxLayers + 1];       // pre-activations, l = 1..L
    float* A[kMaxLayers + 1];       // activations, l = 1..L
    float* Zd[kMaxLayers + 1];      // tangents
    float* Ad[kMaxLayers + 1];
    float* Ab; float* Ab2; float* Adb; float* Zb; float* Zdb;   // [N, max_hidden]
    float* part;                    // [splits, P]
    int splits;
    const int32_t* seg_off;
    int32_t* tile_start;
};

cudaError_t mlp_tiles(const MlpPlan& p, const int32_t* seg_off, int32_t* tile_start, cudaStream_t s, int* launches);
// layers l0 .. L-1 (l0 = 1 when the first layer ran on the tensor cores)
cudaError_t mlp_forward(const MlpPlan& p, const MlpBuffers& b, const float* theta, int64_t N, cudaStream_t s, int* launches,
                        int l0 = 0);
cudaError_t mlp_energy_rows(const MlpPlan& p, const MlpBuffers& b, int64_t N, float* E_rows, cudaStream_t s, int* launches);
// g = dE/dG; with ab1 != nullptr the chain stops at dE/dA_1 (row stride ld[1]), returned in *ab1;
// seeded: b.Ab already holds the output seeds (rows, stride ld[L]) instead of dE/da_L = 1
cudaError_t mlp_input_grad(const MlpPlan& p, const MlpBuffers& b, const float* theta, int64_t N, float* g,
                           cudaStream_t s, int* launches, float** ab1 = nullptr, bool seeded = false);
// BF16 tensor-core networks (mlp_tc.cu): energies and input gradients; ws from tc_workspace_bytes
size_t tc_workspace_bytes(const MlpPlan& p, int64_t N, bool split);
// g16_ready: the descriptor kernel already wrote the BF16 operand rows (tc_g16), else the FP32
// rows b.G are converted first
cudaError_t mlp_bf16_energy_grad(const MlpPlan& p, const MlpBuffers& b, const float* theta, int64_t N, void* ws,
                                 bool split, float* E_rows, float* g, DevStatus* status, cudaStream_t s,
                                 int* launches, bool g16_ready = false);
// the BF16 descriptor operand rows (hi, lo; lo null without split) inside the workspace ws, or
// null when the descriptor width is not a multiple of 8
void tc_g16(const MlpPlan& p, int64_t N, bool split, void* ws, __nv_bfloat16** hi, __nv_bfloat16** lo);
struct WgradTc;
// Parts of the weight-gradient pass: both (default); the forward tangent along wdot only (the
// output tangents land in b.Ad[L]); or the reverse pass only, with the output seeds already in
// b.Ab (energy part) and b.Adb (force part), rows of stride ld[L]
enum MlpGradPart { MLP_GRAD_ALL = 0, MLP_GRAD_TANGENT = 1, MLP_GRAD_REVERSE_SEEDED = 2 };
// tan_tc: the first layer's tangent ran on the tensor cores (tf32_tangent1); wtc (non-null
// ws): every layer's weight gradient on the tensor cores (tf32_wgrad)
cudaError_t mlp_param_grad(const MlpPlan& p, const MlpBuffers& b, const float* theta, int64_t N, const float* wdot,
                           const float* alpha_rows, float* dtheta, cudaStream_t s, int* launches,
                           bool tan_tc = false, const WgradTc* wtc = nullptr, MlpGradPart part = MLP_GRAD_ALL);

// FP32 networks with the first layer on the tensor cores as TF32 hi + lo pairs (mlp_tc.cu).
// Order per call: tf32_prepare, tf32_forward1, mlp_forward(l0 = 1); mlp_input_grad; for
// training tf32_tangent1, then mlp_param_grad(tan_tc, wtc), which calls tf32_wgrad for every
// layer.
// Each of the four products may also stay on the CUDA cores (TF32_* bits below).
enum { TF32_FWD = 1, TF32_INGRAD = 2, TF32_TAN = 4, TF32_WGRAD = 8 };   // TF32_INGRAD: not offered
bool tf32_first_layer_ok(const MlpPlan& p);
// mask: the TF32_* products used in this evaluation (the same value in every call of one evaluation)
size_t tf32_workspace_bytes(const MlpPlan& p, int64_t N, int mask);
cudaError_t tf32_prepare(const MlpPlan& p, const MlpBuffers& b, const float* theta, int64_t N, void* ws, int mask,
                         cudaStream_t s, int* launches);
cudaError_t tf32_forward1(const MlpPlan& p, const MlpBuffers& b, int64_t N, void* ws, int mask, DevStatus* status,
                          cudaStream_t s, int* launches);
cudaError_t tf32_tangent1(const MlpPlan& p, const MlpBuffers& b, int64_t N, void* ws, int mask, const float* Gdot,
                          DevStatus* status, cudaStream_t s, int* launches);
// weight gradient of layer l+1 from b.Zb, b.Zdb (its adjoints) and its inputs A, Ad
cudaError_t tf32_wgrad(const MlpPlan& p, const MlpBuffers& b, int64_t N, void* ws, int mask, int l, const float* A,
                       const float* Ad, float* dtheta, DevStatus* status, cudaStream_t s, int* launches);

// context of the tensor-core weight gradients inside mlp_param_grad (null ws: CUDA cores)
struct WgradTc { void* ws; int mask; DevStatus* status; };

}  // namespace panna
