// Descriptors of a small batch with no device allocation at all.
//
// The ordinary entry points keep their scratch (cell lists, neighbour lists, status word)
// in a workspace that the context allocates with cudaMalloc.  Some callers cannot allow
// that: a host program whose memory pool already owns all of the GPU's memory, or a
// callback (for instance a force call made from inside another code's time step) where
// the host code forbids new device allocations.  panna_descriptors_static serves them:
// its scratch is one file-scope __device__ array of kStaticScratchBytes that every GPU
// which loads this library holds until the process exits.
//
// Host code may not pass the array's symbol to a kernel (on the host it is only a
// stand-in, not a device address), so the first call on each device looks the address up
// with cudaGetSymbolAddress while that device is current and caches it.  All calls share
// the one array: calls that overlap on the GPU race with each other.
#include <math.h>
#include <stdio.h>

#include <mutex>

#include "common.cuh"

using namespace panna;

namespace {

constexpr size_t kStaticScratchBytes = (size_t)32 << 20;   // 32 MiB
constexpr int kStaticMaxCap = 256;                          // neighbour slots per atom, at most
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
void* g_static_addr[kMaxDevices] = {};

struct Carver {
    char* base;
    size_t off = 0;
    template <class T>
    T* take(size_t n)
    {
        off = (off + 255) & ~(size_t)255;
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += (n ? n : 1) * sizeof(T);
        return p;
    }
};

// Neighbour and cell buffers of the descriptor path, carved from `base` (nullptr: sizing).
size_t carve_static(char* base, int64_t N, int64_t C, int cap, Work& w)
{
    Carver a{base};
    w.N = N; w.C = C; w.cap = cap;
    w.cap_cells = 2 * N + C + 1;
    w.status = a.take<DevStatus>(1);
    w.geom = a.take<CfgGeom>(C);
    w.cell_count = a.take<int64_t>(w.cap_cells + 1);
    w.cell_start = a.take<int64_t>(w.cap_cells + 1);
    w.cell_fill = a.take<int32_t>(w.cap_cells);
    w.cell_atoms = a.take<int32_t>(N);
    w.atom_cell = a.take<int32_t>(N);
    w.atom_cfg = a.take<int32_t>(N);
    w.pos_hi = a.take<float4>(N);
    w.pos_lo = a.take<float4>(N);
    w.pos_hi_s = a.take<float4>(N);
    w.pos_lo_s = a.take<float4>(N);
    w.wrap = a.take<int32_t>(3 * N);
    w.scan_tmp = a.take<int64_t>(scan_scratch_elems(w.cap_cells + 1 > N + 1 ? w.cap_cells + 1 : N + 1));
    w.nb_count = a.take<int32_t>(N);
    w.nb_vec = a.take<float4>((size_t)N * cap);
    w.nb_idx = a.take<int2>((size_t)N * cap);
    w.nb_vlo = nullptr;
    w.row_of_atom = nullptr;
    w.atom_of_row = nullptr;
    w.seg_off = nullptr;
    w.blk_counts = nullptr;
    return a.off;
}

panna_status sfail(panna_status st, const char* msg)
{
    set_last_error_message(msg);   // read back through panna_last_error()
    return st;
}

}  // namespace

extern "C" panna_status panna_descriptors_static(const panna_desc_params* p, const panna_system* sys, float* G,
                                                 panna_stream_t stream)
{
    char msg[256];
    if (!p || !sys || !G) return sfail(PANNA_ERR_INVALID_ARG, "null argument");
    bool unsupported = false;
    if (const char* why = desc_params_check(p, &unsupported))
        return sfail(unsupported ? PANNA_ERR_UNSUPPORTED : PANNA_ERR_INVALID_ARG, why);
    const int64_t N = sys->n_atoms, C = sys->n_cfg;
    if (C < 1 || N < 0 || !sys->atom_off || !sys->cell || !sys->pbc || (N > 0 && (!sys->pos || !sys->species)))
        return sfail(PANNA_ERR_INVALID_ARG, "invalid system");
    cudaStream_t s = (cudaStream_t)stream;

    // the largest per-atom neighbour capacity that fits the static array
    Work w{};
    const size_t fixed = carve_static(nullptr, N, C, 0, w);
    if (fixed > kStaticScratchBytes) {
        snprintf(msg, sizeof msg, "%lld atoms in %lld configurations need %zu bytes of scratch before neighbour "
                 "lists; the static buffer holds %zu", (long long)N, (long long)C, fixed, kStaticScratchBytes);
        return sfail(PANNA_ERR_INVALID_ARG, msg);
    }
    const size_t per_slot = sizeof(float4) + sizeof(int2);
    int64_t cap = N > 0 ? (int64_t)((kStaticScratchBytes - fixed - 1024) / ((size_t)N * per_slot)) : kStaticMaxCap;
    if (cap > kStaticMaxCap) cap = kStaticMaxCap;
    if (cap < 8) {
        snprintf(msg, sizeof msg, "%lld atoms exceed the static scratch of %zu bytes (fewer than 8 neighbour "
                 "slots per atom would fit)", (long long)N, kStaticScratchBytes);
        return sfail(PANNA_ERR_INVALID_ARG, msg);
    }

    // device address of the static array, looked up once per device with that device current
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return sfail(PANNA_ERR_CUDA, "no current CUDA device");
    char* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_static_mu);
        if (!g_static_addr[dev]) {
            void* ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
            if (e != cudaSuccess || !ptr) {
                snprintf(msg, sizeof msg, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
                return sfail(PANNA_ERR_CUDA, msg);
            }
            g_static_addr[dev] = ptr;
        }
        base = static_cast<char*>(g_static_addr[dev]);
    }

    // descriptor parameters as the kernels read them
    DescDev d{};
    desc_dev_from_params(p, d);

    // one pass at the largest capacity that fits: a larger one cannot exist
    carve_static(base, N, C, (int)cap, w);
    w.sys = sys;
    int launches = 0;
    // the array keeps the previous call's contents: clear what must start at zero
    cudaError_t e = cudaMemsetAsync(w.status, 0, sizeof(DevStatus), s);
    if (e == cudaSuccess) e = build_neighbors(w, d, s, &launches);
    if (e == cudaSuccess) e = launch_descriptor(w, d, G, nullptr, true, s, &launches);
    DevStatus h{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, w.status, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        snprintf(msg, sizeof msg, "CUDA error: %s", cudaGetErrorString(e));
        return sfail(PANNA_ERR_CUDA, msg);
    }
    if (h.code == 0) return PANNA_OK;
    if (h.code == PANNA_ERR_NEIGHBOR_OVERFLOW) {
        snprintf(msg, sizeof msg, "atom %d has %d neighbours; the static scratch holds %lld per atom for "
                 "%lld atoms", h.bad_index, h.need_cap, (long long)cap, (long long)N);
        return sfail(PANNA_ERR_NEIGHBOR_OVERFLOW, msg);
    }
    snprintf(msg, sizeof msg, "device error %d at index %d", h.code, h.bad_index);
    return sfail((panna_status)h.code, msg);
}
