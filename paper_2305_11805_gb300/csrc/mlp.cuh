// Internal interface of the per-species network kernels.
#pragma once

#include "common.cuh"

namespace panna {

constexpr int kBM = 64, kBN = 64, kBK = 16;
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
cudaError_t mlp_forward(const MlpPlan& p, const MlpBuffers& b, const float* theta, int64_t N, cudaStream_t s, int* launches);
cudaError_t mlp_energy_rows(const MlpPlan& p, const MlpBuffers& b, int64_t N, float* E_rows, cudaStream_t s, int* launches);
cudaError_t mlp_input_grad(const MlpPlan& p, const MlpBuffers& b, const float* theta, int64_t N, float* g,
                           cudaStream_t s, int* launches);
// BF16 tensor-core networks (mlp_tc.cu): energies and input gradients; ws from tc_workspace_bytes
size_t tc_workspace_bytes(const MlpPlan& p, int64_t N, bool split);
cudaError_t mlp_bf16_energy_grad(const MlpPlan& p, const MlpBuffers& b, const float* theta, int64_t N, void* ws,
                                 bool split, float* E_rows, float* g, DevStatus* status, cudaStream_t s,
                                 int* launches);
cudaError_t mlp_param_grad(const MlpPlan& p, const MlpBuffers& b, const float* theta, int64_t N, const float* wdot,
                           const float* alpha_rows, float* dtheta, cudaStream_t s, int* launches);

}  // namespace panna
