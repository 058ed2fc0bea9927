// Convolution forward for callers that cannot allocate device memory.
//
// sevennet_conv_forward_dev needs two per-edge scratch arrays (the receiver of
// every edge and the edge vector with its length) and takes them from
// cudaMallocAsync on each call.  Some callers must not allocate at that point:
// code that runs under a fixed memory plan decided up front, code that must
// not risk the implicit device synchronisation an allocation or free can
// cause, or code that may not re-enter the allocator at all.  This variant
// keeps the scratch in one file-scope device array instead, so the call itself
// allocates and frees nothing.
//
// The array holds at most NOALLOC_MAX_EDGES edges (5 MiB).  Every GPU that
// loads the library keeps it until the process exits.  All calls share it, so
// two calls whose kernels overlap on the GPU race on it; the caller must order
// them (one stream, or events).
#include "internal.h"

#include <mutex>

namespace sn {

constexpr int64_t NOALLOC_MAX_EDGES = 1 << 18;                         // 262,144 edges
constexpr size_t NOALLOC_GEOM_BYTES = (size_t)NOALLOC_MAX_EDGES * sizeof(float4);
constexpr size_t NOALLOC_BYTES = NOALLOC_GEOM_BYTES + (size_t)NOALLOC_MAX_EDGES * sizeof(int);

// [0, NOALLOC_GEOM_BYTES): float4 (d, |d|) per edge; then int receiver per edge.
static __device__ __align__(256) unsigned char g_conv_scratch[NOALLOC_BYTES];

// Host code cannot use g_conv_scratch as a pointer (it is a host-side
// stand-in); its device address is looked up once per device.
static std::mutex g_scratch_mu;
static void* g_scratch_addr[64] = {};

static sevennet_status scratch_address(int device, void** out) {
    SN_CHECK(device >= 0 && device < 64, SEVENNET_EINVAL, "device %d out of range", device);
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        SN_CUDA(cudaGetSymbolAddress(&p, g_conv_scratch));
        g_scratch_addr[device] = p;
    }
    *out = g_scratch_addr[device];
    return SEVENNET_OK;
}

// Receiver of every edge and (d, |d|).  The clamp keeps this kernel's own
// writes inside [0, n_edges); it does not make an invalid CSR safe: the
// convolution walks the edges by the caller's row_ptr, which must be a valid
// CSR with row_ptr[n_atoms] == n_edges (as the header states).
__global__ void noalloc_prepare_kernel(int64_t n_atoms, int64_t n_edges, const int* __restrict__ row_ptr,
                                       const float* __restrict__ d, int* __restrict__ dst,
                                       float4* __restrict__ geom) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_atoms) {
        const int64_t e0 = max((int64_t)row_ptr[i], (int64_t)0);
        const int64_t e1 = min((int64_t)row_ptr[i + 1], n_edges);
        for (int64_t e = e0; e < e1; ++e) dst[e] = (int)i;
    }
    if (i < n_edges) {
        const float x = d[i * 3], y = d[i * 3 + 1], z = d[i * 3 + 2];
        geom[i] = make_float4(x, y, z, sqrtf(x * x + y * y + z * z));
    }
}

}  // namespace sn

using namespace sn;

extern "C" sevennet_status sevennet_conv_forward_noalloc(sevennet_model* M, int32_t layer, int64_t n_atoms,
                                                         int64_t n_edges, const int32_t* row_ptr,
                                                         const int32_t* src, const float* d, const float* x,
                                                         float* m_out, sevennet_precision prec, void* stream) {
    SN_CHECK(M && layer >= 0 && layer < M->T && n_atoms >= 0 && n_edges >= 0, SEVENNET_EINVAL, "bad argument");
    SN_CHECK(row_ptr && x && m_out && (n_edges == 0 || (src && d)), SEVENNET_EINVAL, "NULL argument");
    SN_CHECK(n_edges <= NOALLOC_MAX_EDGES, SEVENNET_EINVAL,
             "sevennet_conv_forward_noalloc: %lld edges exceed its fixed scratch of %lld edges; "
             "use sevennet_conv_forward_dev", (long long)n_edges, (long long)NOALLOC_MAX_EDGES);
    SN_CHECK(prec == SEVENNET_FP32 || prec == SEVENNET_BF16, SEVENNET_EINVAL, "unknown precision");
    SN_ENTER(M->device);
    void* base = nullptr;
    SN_TRY(scratch_address(M->device, &base));
    float4* geom = static_cast<float4*>(base);
    int* dst = reinterpret_cast<int*>(static_cast<unsigned char*>(base) + NOALLOC_GEOM_BYTES);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t n = std::max(n_atoms, n_edges);
    if (n > 0)
        noalloc_prepare_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n_atoms, n_edges, row_ptr, d, dst, geom);
    launch_conv_fwd(M->layers[layer], M->H, prec, n_atoms, n_edges, row_ptr, dst, src, geom, x, m_out, st);
    SN_CUDA(cudaGetLastError());
    return SEVENNET_OK;
}
