// Internal declarations shared by the libppgmres translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>
#include <vector>

#include "../../include/ppgmres.h"

namespace ppg {

// ---------------------------------------------------------------------------
// Errors and bookkeeping
// ---------------------------------------------------------------------------

void set_cuda_error(cudaError_t e, const char* where);
extern thread_local int64_t g_launches;   // kernels launched by this thread

#define PPG_CUDA(call)                                                    \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) {                                          \
            ::ppg::set_cuda_error(e_, #call);                             \
            return PPG_ERR_CUDA;                                          \
        }                                                                 \
    } while (0)

#define PPG_TRY(expr)                                                     \
    do {                                                                  \
        int32_t rc_ = (expr);                                             \
        if (rc_ < 0) return rc_;                                          \
    } while (0)

int32_t check_launch(const char* where);

// Argument checks shared by the entry points: a CSR descriptor (dtype
// PPG_F64 or PPG_F32; dtype_required < 0 accepts either) and a root list
// (finite values, no zero root, conjugate pairs adjacent and exact).
int32_t check_csr(const ppg_csr* A, int dtype_required);
int32_t check_roots(const ppg_roots* r);

// Programmatic dependent launch.  A kernel launched with launch_pdl may
// start while the previous kernel in the stream finishes; it must call
// PPG_PDL_WAIT() before touching any global data that earlier work writes
// (and before writing anything earlier work reads).  PPG_PDL_TRIGGER() lets
// the next kernel start launching.
#define PPG_PDL_TRIGGER() asm volatile("griddepcontrol.launch_dependents;")
#define PPG_PDL_WAIT() asm volatile("griddepcontrol.wait;" ::: "memory")

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// One stream-ordered scratch allocation carved into 256-byte aligned pieces.
struct Arena {
    size_t bytes = 0;
    char* base = nullptr;
    struct Req { void** out; size_t bytes; };
    std::vector<Req> reqs;
    template <typename T>
    void add(T** out, size_t count) {
        reqs.push_back({(void**)out, count * sizeof(T)});
    }
    int32_t alloc(cudaStream_t s) {
        size_t off = 0;
        for (auto& r : reqs) off += (r.bytes + 255) / 256 * 256;
        bytes = off;
        if (bytes == 0) return PPG_OK;
        cudaError_t e = cudaMallocAsync((void**)&base, bytes, s);
        if (e != cudaSuccess) {
            set_cuda_error(e, "cudaMallocAsync");
            cudaGetLastError();
            return PPG_ERR_NOMEM;
        }
        off = 0;
        for (auto& r : reqs) {
            *r.out = base + off;
            off += (r.bytes + 255) / 256 * 256;
        }
        return PPG_OK;
    }
    void release(cudaStream_t s) {
        if (base) cudaFreeAsync(base, s);
        base = nullptr;
    }
};

// Keep freed scratch cached in the device's default pool (once per device).
int32_t setup_device_pool();

// Streaming multiprocessors of the current device (queried once per device).
int device_sm_count();
// Grid cap for grid-stride elementwise kernels: `per_sm` CTAs per SM.
inline int grid_cap(int per_sm) { return per_sm * device_sm_count(); }

// ---------------------------------------------------------------------------
// Fused SpMV-root step (one pass over A per root; Algorithms 1 and 3)
// ---------------------------------------------------------------------------

enum StepOp : int {
    OP_SPMV = 0,      // o0 = A x
    OP_RESID = 1,     // o0 = a0 - A x, part[block] = sum o0^2
    OP_PHI_REAL = 2,  // pi' = a0 - c1 (A x)               (x = a0 = pi)
    OP_PHI_PAIR2 = 3, // pi' = a1 + c2 (A x - c1 a0)       (x = a0 = prod, a1 = pi)
    OP_P_REAL = 4,    // p' = a1 + c1 a0 ; prod' = a0 - c1 (A x)   (x = a0 = prod)
    OP_P_PAIR1 = 5,   // tmp = c1 a0 - A x ; p' = a1 + c2 tmp      (x = a0 = prod)
    OP_P_PAIR2 = 6,   // prod' = a0 - c2 (A x)                     (x = tmp, a0 = prod)
};

enum StepFlag : int {
    F_FINAL = 1,   // PHI_*: o0 = a2 - pi' ; P_REAL: o0 = p' + c3 prod' ;
                   // P_PAIR2: o0 = a1 + c3 prod'
    F_PZERO = 2,   // P_*: the accumulator p starts at zero (a1 not read)
    F_NO_O1 = 4,   // P_PAIR1: tmp not needed afterwards
    F_KEEP_A = 8,  // copy A with an L2 evict-last hint (A and the vectors fit in L2)
};

template <typename T>
struct StepArgs {
    const int32_t* rowptr;
    const int32_t* colind;
    const T* vals;
    int32_t n;
    const T* x;
    const T* a0;
    const T* a1;
    const T* a2;
    T* o0;
    T* o1;
    T c1, c2, c3;
    int32_t flags;
    double* part;
    int32_t pf_ahead;   // tiles ahead to prefetch into L2 (set by launch_step)
    int32_t keep_rows;  // rows [0, keep_rows) stage their nonzeros with an L2
                        // evict-last hint (a chain over a matrix too large
                        // for L2 keeps its leading rows resident)
};

// Systems of at most DIRECT_MAX_N rows take the direct-read variant of the
// step (one row per thread, no staging round: latency, not bytes, sets the
// time of a step that is a handful of CTAs); the results are identical.
constexpr int32_t DIRECT_MAX_N = 32768;

// launch one fused step; returns the number of blocks (= partial sums for
// OP_RESID) or a negative status
template <typename T>
int32_t launch_step(int op, const StepArgs<T>& a, cudaStream_t s);

// a root step with the operator product precomputed in prodv (composite
// operators); returns the grid (= partial sums for OP_RESID) or a status
template <typename T>
int32_t launch_ew_step(int op, const StepArgs<T>& a, const T* prodv, cudaStream_t s);

// F_KEEP_A when the matrix plus `nvec` work vectors fit comfortably in L2.
// The first such request reserves an L2 set-aside for the matrix (a limit of
// the process's context on the current device); with may_reserve = false
// nothing is reserved and F_KEEP_A is returned only if a set-aside large
// enough already exists on this device.
// keep_rows (root-step chains only): for a matrix that does not fit, the
// number of leading rows whose nonzeros a chain holds in an L2 set-aside of
// about 48 MB, which is set to that size (with may_reserve; otherwise the
// set-aside in place, if any, is used); 0 without a set-aside.  Other callers
// pass nullptr and leave the set-aside as it is.
int keep_a_flag(int64_t n, int64_t nnz, int elem, int nvec, bool may_reserve = true,
                int32_t* keep_rows = nullptr);

// at least the partial sums any residual step of n rows writes (one per CTA)
int32_t spmv_grid_blocks(int32_t n);

// algorithmic bytes of one fused step
double step_bytes(int op, int flags, int64_t n, int64_t nnz, int elem);

// ---------------------------------------------------------------------------
// Root-step plans (host side; built once per roots and reused)
// ---------------------------------------------------------------------------

enum BufId : int { B_IN = 0, B_OUT = 1, B_A = 2, B_B = 3, B_C = 4, B_P = 5, B_NONE = -1 };

struct Step {
    int op;
    int flags;
    double c1, c2, c3;
    int x, a0, a1, a2, o0, o1;   // BufId
};

// Algorithm 1: in = v, out = phi(A) v (or pi(A) v when want_pi)
std::vector<Step> plan_phi(const double* re, const double* im, int d, bool want_pi);
// Algorithm 3: in = v; accumulator B_P (starts at zero unless accumulate)
std::vector<Step> plan_p(const double* re, const double* im, int d, bool accumulate);

struct Buffers {
    void* ptr[6];
};

// reserve_l2 = false: never change the context's L2 set-aside (see keep_a_flag)
template <typename T>
int32_t run_plan(const std::vector<Step>& plan, const int32_t* rowptr,
                 const int32_t* colind, const T* vals, int32_t n, int64_t nnz,
                 const Buffers& bufs, cudaStream_t s, double* bytes_out,
                 bool reserve_l2 = true);

// ---------------------------------------------------------------------------
// Multi-root fused sweep (sweep.cu): Algorithm 3 on a plan's reordered FP32
// matrix with each conjugate pair in one pass
// ---------------------------------------------------------------------------

int32_t sweep_run_chain(const ppg_sweep_plan* P, const std::vector<Step>& plan,
                        const Buffers& bufs, cudaStream_t s);
// y = x[perm] (x FP64 when x_f64, else FP32), into the plan's ordering
int32_t sweep_gather(const ppg_sweep_plan* P, const void* x, bool x_f64, float* y,
                     cudaStream_t s);
// y[perm] = x, back to the original ordering
int32_t sweep_scatter(const ppg_sweep_plan* P, const float* x, float* y, cudaStream_t s);
// algorithmic bytes and launches of a chain run by sweep_run_chain
double sweep_chain_bytes(const ppg_sweep_plan* P, const std::vector<Step>& plan);
int64_t sweep_chain_launches(const ppg_sweep_plan* P, const std::vector<Step>& plan);
int32_t sweep_plan_n(const ppg_sweep_plan* P);

// ---------------------------------------------------------------------------
// Orthogonalisation and small dense kernels
// ---------------------------------------------------------------------------

struct OrthoWs {
    double* part;       // [ortho_part_doubles(grid)]
    unsigned* counter;  // [4] zero-initialised: [0..2] self-resetting CTA
                        // counters of the passes, [3] error flag (a staging
                        // wait of the fused pass gave up)
    double* h1;         // [MAXC + 2]
    double* h2;         // [MAXC + 2]
    double* nrm;        // [4]
    int grid;
};

constexpr int ORTHO_MAXC = 256;   // max columns (m + 1)

int ortho_grid(int32_t n);
size_t ortho_part_doubles(int grid);

// h_out = V[:, :ncol]^T w  (+ w.w in h_out[ncol] if with_self)
int32_t launch_cgs_dot(const double* V, int64_t ldv, int ncol, const double* w,
                       int32_t n, bool with_self, double* h_out,
                       const OrthoWs& ws, cudaStream_t s);
// w -= V hin ; with_norm: nrm_out[0] = w.w afterwards
int32_t launch_cgs_update(const double* V, int64_t ldv, int ncol, double* w,
                          int32_t n, const double* hin, bool with_norm, double* nrm_out,
                          const OrthoWs& ws, cudaStream_t s);

// w -= V h1 and h2_out = V^T w (the updated w) in one pass: CGS2 passes 2
// and 3 fused.  Needs cgs_fused_ok(V, ldv, ncol, w): V and w 16-byte
// aligned, ldv a multiple of 64, w a column of the same padded basis (ldv
// rows readable), ncol <= 56.
bool cgs_fused_ok(const double* V, int64_t ldv, int ncol, const double* w);
int32_t launch_cgs_sub_dot(const double* V, int64_t ldv, int ncol, double* w, int32_t n,
                           const double* h1, double* h2_out, const OrthoWs& ws,
                           cudaStream_t s);

struct GmresState {   // device, one per solve
    double* R;        // (m+1) x m column-major, rotated Hessenberg
    double* Hraw;     // (m+1) x m column-major, un-rotated (build_poly)
    double* cs;       // [m]
    double* sn;       // [m]
    double* g;        // [m+1]
    double* y;        // [m]
    double* scal;     // [8]: 0 est, 1 h_{j+1,j}, 2 inv_h, 3 beta, 4 inv_beta,
                      //      5 breakdown flag, 6 first breakdown step, 7 spare
};

// Hessenberg column j from h1 + h2 and nrm (w.w); givens = apply rotations
// and update g; breakdown_rtol > 0 compares h_{j+1,j} with
// breakdown_rtol * sqrt(w0sq) where w0sq = h1[ncol]
int32_t launch_finish_column(const GmresState& st, int ldh, int j,
                             const double* h1, const double* h2,
                             const double* nrm, bool givens, double bnorm,
                             double breakdown_rtol, cudaStream_t s);
int32_t launch_scale(const double* x, double* y, int32_t n, const double* scal_ptr,
                     cudaStream_t s);
int32_t launch_backsolve(const GmresState& st, int ldh, int k, cudaStream_t s);
template <typename TV>
int32_t launch_gemv_acc(const TV* V, int64_t ldv, int k, const double* y,
                        double* out, int32_t n, bool accumulate, cudaStream_t s);
int32_t launch_reduce_norm(const double* part, int nparts, double* scal,
                           double* g0, cudaStream_t s);
int32_t launch_norm2_part(const double* x, int32_t n, double* part,
                          cudaStream_t s, int* nparts);
int32_t launch_diff_norm2_part(const double* a, const double* b, int32_t n,
                               double* part, cudaStream_t s, int* nparts);
int32_t launch_cast_f64_f32(const double* x, float* y, int32_t n, cudaStream_t s);
int32_t launch_cast_f32_f64(const float* x, double* y, int32_t n, cudaStream_t s);
int32_t launch_fill(double* x, double v, int32_t n, cudaStream_t s);
template <typename T>
int32_t launch_axpby(T a, const T* x, T b, const T* y, T* out, int32_t n,
                     cudaStream_t s);

// transpose / adjoint
int32_t launch_transpose(const ppg_csr* A, int32_t* rowptr_t, int32_t* colind_t,
                         void* vals_t, int32_t* perm, int32_t* work,
                         cudaStream_t s);
int32_t launch_adjoint_grad(const ppg_csr* A, const double* lam,
                            const double* x, double* gvals, cudaStream_t s);

// ---------------------------------------------------------------------------
// Host polynomial construction (host_poly.cpp)
// ---------------------------------------------------------------------------

int32_t host_harmonic_ritz(const double* Hbar, int ldh, int d, double* re, double* im);
int32_t host_leja(int k, const double* re, const double* im, double* ro, double* io);
int32_t host_add_roots(int k, const double* re, const double* im, double thr,
                       double step, ppg_roots* out);

}  // namespace ppg
