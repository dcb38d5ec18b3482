// rlsq_trsv_noalloc: the sync-free triangular solve with its scratch memory in
// a file-scope device array instead of buffers that the library allocates.
//
// Who needs this: callers that must not allocate device memory while they
// run, for instance a latency-critical serving loop (cudaMalloc can stall
// the device while it runs) or a process whose free device memory is already
// reserved by another allocator.  They still pass their own input and output
// buffers; the solve's working memory -- per-row ready flags, the chunk
// ticket counter and the error word -- comes from the array below, which
// every GPU that loads the library holds until the process exits.
#include <mutex>

#include <cuda.h>

#include "common.h"

// The scratch memory of rlsq_trsv_noalloc (8 MiB + 512 B per device).
static __device__ __align__(256) int32_t g_trsv_scratch[128 + RLSQ_NOALLOC_MAX_ROWS];

namespace rlsq {

namespace {

// Layout of the scratch array, in 32-bit words:
//   [0, 64)      a solver state block (only `done`, `apply_count`, `error` are used)
//   [64, 128)    ticket counters
//   [128, 128+n) ready flags, one per row
constexpr int kStateWords = 64;
constexpr int kTicketWords = kMaxSlots;
constexpr int kHeaderWords = kStateWords + kTicketWords;
static_assert(sizeof(LsmrState) <= kStateWords * sizeof(int32_t), "state block too small");
static_assert(kHeaderWords == 128, "header size");

std::mutex g_mutex;
constexpr int kMaxDevices = 64;
// The array's device address, per device ordinal, with the id of the CUDA
// context it was looked up in: a device reset (cudaDeviceReset) ends that
// context, the next one gets a new id, and the address is looked up again.
struct ScratchAddr {
    unsigned long long ctx_id = 0;
    void* addr = nullptr;
};
ScratchAddr g_scratch_addr[kMaxDevices];

using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// cuCtxGetId through the runtime's driver entry point (no link to libcuda).
unsigned long long current_context_id() {
    static CtxGetIdFn fn = []() -> CtxGetIdFn {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<CtxGetIdFn>(f);
    }();
    if (!fn) throw ApiError(RLSQ_ERR_CUDA, "cuCtxGetId is not available from the driver");
    unsigned long long id = 0;
    if (fn(nullptr, &id) != CUDA_SUCCESS) throw ApiError(RLSQ_ERR_CUDA, "cuCtxGetId failed");
    return id;
}

// Device address of g_trsv_scratch on the current device, looked up once per
// device and context.  (In host code the symbol's name is only a stand-in;
// its device address comes from cudaGetSymbolAddress.)
int32_t* scratch_on_current_device() {
    int dev = 0;
    RLSQ_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) throw ApiError(RLSQ_ERR_ARG, "device ordinal out of range");
    RLSQ_CUDA(cudaSetDevice(dev));  // makes the device's primary context current on this thread
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lock(g_mutex);
    ScratchAddr& a = g_scratch_addr[dev];
    if (!a.addr || a.ctx_id != ctx) {
        void* p = nullptr;
        RLSQ_CUDA(cudaGetSymbolAddress(&p, g_trsv_scratch));
        a.addr = p;
        a.ctx_id = ctx;
    }
    return static_cast<int32_t*>(a.addr);
}

template <class F>
void with_lanes(int G, F&& f) {
    switch (G) {
        case 1: f(std::integral_constant<int, 1>{}); break;
        case 2: f(std::integral_constant<int, 2>{}); break;
        case 4: f(std::integral_constant<int, 4>{}); break;
        case 8: f(std::integral_constant<int, 8>{}); break;
        case 16: f(std::integral_constant<int, 16>{}); break;
        default: f(std::integral_constant<int, 32>{}); break;
    }
}

}  // namespace
}  // namespace rlsq

using namespace rlsq;

extern "C" int rlsq_trsv_noalloc(rlsq_problem h, int32_t which, const double* b, double* x, void* stream) {
    return guarded([&]() -> int {
        if (!h || !b || !x) throw ApiError(RLSQ_ERR_ARG, "null argument");
        if (which < 0 || which > 3) throw ApiError(RLSQ_ERR_ARG, "bad system id");
        if (!h->factored) throw ApiError(RLSQ_ERR_NOT_FACTORED, "rlsq_factor has not succeeded");
        if (h->precision != RLSQ_PREC_FP64)
            throw ApiError(RLSQ_ERR_ARG, "rlsq_trsv_noalloc needs a problem factored with RLSQ_PREC_FP64");
        if (h->n > RLSQ_NOALLOC_MAX_ROWS)
            throw ApiError(RLSQ_ERR_SHAPE, "rlsq_trsv_noalloc handles at most RLSQ_NOALLOC_MAX_ROWS (" +
                                               std::to_string(RLSQ_NOALLOC_MAX_ROWS) + ") rows; this problem has " +
                                               std::to_string(h->n));
        int dev = 0;
        RLSQ_CUDA(cudaGetDevice(&dev));
        if (dev != h->device) throw ApiError(RLSQ_ERR_ARG, "the problem lives on another device");
        int32_t* base = scratch_on_current_device();
        LsmrState* S = reinterpret_cast<LsmrState*>(base);
        unsigned* tickets = reinterpret_cast<unsigned*>(base + kStateWords);
        int* flags = base + kHeaderWords;
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        const int n = static_cast<int>(h->n);
        // the array keeps the previous call's contents: clear state, tickets, flags
        RLSQ_CUDA(cudaMemsetAsync(base, 0, sizeof(int32_t) * (kHeaderWords + static_cast<size_t>(n)), st));
        const Tri<double> tri = h->f64.tview(which);
        const Rhs<double> rhs{b, nullptr, nullptr};
        with_lanes(h->map.G_tri[which], [&](auto g) {
            constexpr int GG = decltype(g)::value;
            constexpr int ROUNDS = 4;
            auto kern = k_trsv_syncfree<double, GG, RHS_VEC, ROUNDS>;
            int occ = 0;
            RLSQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kBlock, 0));
            const int chunk_rows = (kBlock / GG) * ROUNDS;
            const int chunks = (n + chunk_rows - 1) / chunk_rows;
            const int grid = std::max(1, std::min(chunks, std::max(1, occ) * h->num_sms));
            kern<<<grid, kBlock, 0, st>>>(tri, rhs, x, flags, 0, tickets, S, &base[offsetof(LsmrState, error) / 4]);
        });
        RLSQ_CUDA(cudaGetLastError());
        int err = 0;
        RLSQ_CUDA(cudaMemcpyAsync(&err, &base[offsetof(LsmrState, error) / 4], sizeof(int),
                                  cudaMemcpyDeviceToHost, st));
        RLSQ_CUDA(cudaStreamSynchronize(st));
        if (err) throw ApiError(RLSQ_ERR_DEVICE_TIMEOUT, "a sync-free triangular solve timed out");
        return RLSQ_OK;
    });
}
