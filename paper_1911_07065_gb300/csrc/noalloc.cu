// y = p(A) v (the same fused SpMV-root chain as ppg_apply_poly) for callers
// that cannot allocate device memory: its work vectors live in a fixed
// array compiled into this library instead of coming from cudaMallocAsync.
//
// Why: some callers must not allocate at call time -- their device memory
// is already reserved by another allocator (a framework's caching allocator
// that holds the whole GPU), or an allocation or free would synchronise the
// device or could fail under memory pressure in the middle of their work.
//
// The array is file-scope device memory: every GPU that loads the library
// holds it (3 * PPG_NOALLOC_MAX_N doubles, 24 MiB) until the process exits.
// Host code must not pass the array's name to a kernel (on the host it is
// only a stand-in for the device symbol); its device address is looked up
// once per device with cudaGetSymbolAddress, with that device current, on
// the first call made on that device.  Apart from that lookup the entry point
// changes no state of the context: unlike ppg_apply_poly it never reserves an
// L2 set-aside for the matrix.
#include <mutex>

#include "ppg_common.cuh"

namespace ppg {

namespace {

// three work vectors of up to PPG_NOALLOC_MAX_N entries: the two
// alternating "prod" buffers of Algorithm 3 and the conjugate-pair
// temporary.  Slots are PPG_NOALLOC_MAX_N doubles apart for either dtype.
static __device__ __align__(256) double g_noalloc_scratch[3 * (size_t)PPG_NOALLOC_MAX_N];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// device address of g_noalloc_scratch on the current device (set up on the
// first call made on that device).  That first call must not be made while
// `s` is being captured into a graph: the lookup may load the library's
// device code, which a capture does not allow, so it is refused instead.
int32_t scratch_address(cudaStream_t s, void** out) {
    int dev = 0;
    PPG_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return PPG_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (g_scratch_addr[dev] == nullptr) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        PPG_CUDA(cudaStreamIsCapturing(s, &cs));
        if (cs != cudaStreamCaptureStatusNone) return PPG_ERR_ARG;
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            set_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
            return PPG_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return PPG_OK;
}

}  // namespace

}  // namespace ppg

using namespace ppg;

extern "C" int32_t ppg_apply_poly_noalloc(const ppg_csr* A, const ppg_roots* r, const void* v,
                                          void* y, void* stream) {
    // the same argument checks as ppg_apply_poly
    PPG_TRY(check_csr(A, -1));
    PPG_TRY(check_roots(r));
    if (!v || !y || v == y) return PPG_ERR_ARG;
    if (A->n > PPG_NOALLOC_MAX_N) return PPG_ERR_TOO_LARGE;
    cudaStream_t s = (cudaStream_t)stream;
    void* base = nullptr;
    PPG_TRY(scratch_address(s, &base));
    // Nothing in the array has to start at zero: within one call every slot
    // is written before it is read (the accumulator is the caller's y).
    const size_t slot = (size_t)PPG_NOALLOC_MAX_N * sizeof(double);
    Buffers bufs{};
    bufs.ptr[B_IN] = const_cast<void*>(v);
    bufs.ptr[B_OUT] = y;
    bufs.ptr[B_P] = y;
    bufs.ptr[B_A] = (char*)base;
    bufs.ptr[B_B] = (char*)base + slot;
    bufs.ptr[B_C] = (char*)base + 2 * slot;
    const std::vector<Step> plan = plan_p(r->re, r->im, r->n_total, false);
    // reserve_l2 = false: this entry point leaves the context's L2
    // set-aside as it finds it (the cache hint changes no result)
    if (A->dtype == PPG_F64)
        return run_plan<double>(plan, A->rowptr, A->colind, (const double*)A->vals, A->n,
                                A->nnz, bufs, s, nullptr, false);
    return run_plan<float>(plan, A->rowptr, A->colind, (const float*)A->vals, A->n, A->nnz,
                           bufs, s, nullptr, false);
}
