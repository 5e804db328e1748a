// C ABI of libppgmres: plans that turn a root list into a chain of fused
// SpMV-root launches (Algorithms 1 and 3), the polynomial construction
// (Algorithm 4 step 1) and restarted (F)GMRES around the chains (Algorithm 4
// step 2, plus the FP32-inner flexible form), the stability check of
// Section 3.5 and the adjoint helpers.
#include <atomic>
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "ppg_common.cuh"

namespace ppg {

thread_local int64_t g_launches = 0;
static thread_local char g_cuda_err[256] = "";

void set_cuda_error(cudaError_t e, const char* where) {
    snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", where, cudaGetErrorString(e));
}

int32_t check_launch(const char* where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_cuda_error(e, where);
        return PPG_ERR_CUDA;
    }
    return PPG_OK;
}

// ---------------------------------------------------------------------------
// Plans
// ---------------------------------------------------------------------------

constexpr int OP_AXPY = -1;   // elementwise: P = c1 * in (+ P)

static int other_buf(int c) { return c == B_A ? B_B : B_A; }

std::vector<Step> plan_phi(const double* re, const double* im, int d, bool want_pi) {
    std::vector<Step> P;
    int cur = B_IN;
    int i = 0;
    while (i < d) {
        const bool real = im[i] == 0.0;
        const bool last = real ? (i == d - 1) : (i + 1 == d - 1);
        const int dst = last ? B_OUT : other_buf(cur);
        const bool fin = last && !want_pi;
        if (real) {
            P.push_back({OP_PHI_REAL, fin ? F_FINAL : 0, 1.0 / re[i], 0.0, 0.0, cur, cur,
                         B_NONE, fin ? B_IN : B_NONE, dst, B_NONE});
            i += 1;
        } else {
            const double a = re[i], b = im[i];
            P.push_back({OP_SPMV, 0, 0.0, 0.0, 0.0, cur, B_NONE, B_NONE, B_NONE, B_C, B_NONE});
            P.push_back({OP_PHI_PAIR2, fin ? F_FINAL : 0, 2.0 * a, 1.0 / (a * a + b * b), 0.0,
                         B_C, B_C, cur, fin ? B_IN : B_NONE, dst, B_NONE});
            i += 2;
        }
        cur = dst;
    }
    return P;
}

std::vector<Step> plan_p(const double* re, const double* im, int d, bool accumulate) {
    std::vector<Step> P;
    bool pzero = !accumulate;
    if (d == 1) {
        P.push_back({OP_AXPY, pzero ? F_PZERO : 0, 1.0 / re[0], 0.0, 0.0, B_IN, B_NONE,
                     pzero ? B_NONE : B_P, B_NONE, B_P, B_NONE});
        return P;
    }
    const bool final_real = im[d - 1] == 0.0;
    int prod = B_IN;
    int i = 0;
    while (i < d - 1) {
        const int pz = pzero ? F_PZERO : 0;
        const int a1 = pzero ? B_NONE : B_P;
        if (im[i] == 0.0) {
            const bool fuse = (i == d - 2) && final_real;
            const int dst = fuse ? B_NONE : other_buf(prod);
            P.push_back({OP_P_REAL, pz | (fuse ? F_FINAL : 0), 1.0 / re[i], 0.0,
                         fuse ? 1.0 / re[d - 1] : 0.0, prod, prod, a1, B_NONE, B_P, dst});
            prod = dst;
            i += 1;
        } else {
            const double a = re[i], b = im[i];
            const double c2 = 1.0 / (a * a + b * b);
            const bool lastpair = (i + 1 == d - 1);
            P.push_back({OP_P_PAIR1, pz | (lastpair ? F_NO_O1 : 0), 2.0 * a, c2, 0.0, prod,
                         prod, a1, B_NONE, B_P, lastpair ? B_NONE : B_C});
            if (i <= d - 3) {
                const bool fuse = (i + 2 == d - 1) && final_real;
                if (fuse) {
                    P.push_back({OP_P_PAIR2, F_FINAL, 0.0, c2, 1.0 / re[d - 1], B_C, prod, B_P,
                                 B_NONE, B_P, B_NONE});
                } else {
                    const int dst = other_buf(prod);
                    P.push_back({OP_P_PAIR2, 0, 0.0, c2, 0.0, B_C, prod, B_NONE, B_NONE, dst,
                                 B_NONE});
                    prod = dst;
                }
            }
            i += 2;
        }
        pzero = false;
    }
    return P;
}

template <typename T>
static const T* cbuf(const Buffers& b, int id) {
    return id < 0 ? nullptr : (const T*)b.ptr[id];
}
template <typename T>
static T* mbuf(const Buffers& b, int id) {
    return id < 0 ? nullptr : (T*)b.ptr[id];
}

template <typename T>
static int32_t run_steps(const std::vector<Step>& plan, int i0, int i1, const int32_t* rowptr,
                         const int32_t* colind, const T* vals, int32_t n, int64_t nnz,
                         const Buffers& bufs, cudaStream_t s, double* bytes_out,
                         bool reserve_l2 = true);

template <typename T>
int32_t run_plan(const std::vector<Step>& plan, const int32_t* rowptr, const int32_t* colind,
                 const T* vals, int32_t n, int64_t nnz, const Buffers& bufs, cudaStream_t s,
                 double* bytes_out, bool reserve_l2) {
    return run_steps<T>(plan, 0, (int)plan.size(), rowptr, colind, vals, n, nnz, bufs, s,
                        bytes_out, reserve_l2);
}

// steps [i0, i1) of a plan, in order
template <typename T>
static int32_t run_steps(const std::vector<Step>& plan, int i0, int i1, const int32_t* rowptr,
                         const int32_t* colind, const T* vals, int32_t n, int64_t nnz,
                         const Buffers& bufs, cudaStream_t s, double* bytes_out,
                         bool reserve_l2) {
    double bytes = 0.0;
    int32_t keep_rows = 0;
    const int keep = keep_a_flag(n, nnz, (int)sizeof(T), 3, reserve_l2, &keep_rows);
    for (int i = i0; i < i1; ++i) {
        const Step& st = plan[(size_t)i];
        if (st.op == OP_AXPY) {
            const bool pz = st.flags & F_PZERO;
            PPG_TRY(launch_axpby<T>((T)st.c1, cbuf<T>(bufs, st.x), pz ? T(0) : T(1),
                                    pz ? nullptr : cbuf<T>(bufs, B_P), mbuf<T>(bufs, B_P), n, s));
            bytes += (double)sizeof(T) * n * (pz ? 2 : 3);
            continue;
        }
        StepArgs<T> a{};
        a.rowptr = rowptr;
        a.colind = colind;
        a.vals = vals;
        a.n = n;
        a.x = cbuf<T>(bufs, st.x);
        a.a0 = cbuf<T>(bufs, st.a0);
        a.a1 = cbuf<T>(bufs, st.a1);
        a.a2 = cbuf<T>(bufs, st.a2);
        a.o0 = mbuf<T>(bufs, st.o0);
        a.o1 = mbuf<T>(bufs, st.o1);
        a.c1 = (T)st.c1;
        a.c2 = (T)st.c2;
        a.c3 = (T)st.c3;
        a.flags = st.flags | keep;
        a.keep_rows = keep_rows;
        a.part = nullptr;
        int32_t rc = launch_step<T>(st.op, a, s);
        if (rc < 0) return rc;
        bytes += step_bytes(st.op, st.flags, n, nnz, (int)sizeof(T));
    }
    if (bytes_out) *bytes_out = bytes;
    return PPG_OK;
}

template int32_t run_plan<double>(const std::vector<Step>&, const int32_t*, const int32_t*,
                                  const double*, int32_t, int64_t, const Buffers&, cudaStream_t,
                                  double*, bool);
template int32_t run_plan<float>(const std::vector<Step>&, const int32_t*, const int32_t*,
                                 const float*, int32_t, int64_t, const Buffers&, cudaStream_t,
                                 double*, bool);

// ---------------------------------------------------------------------------
// Workspace: one stream-ordered allocation carved into aligned pieces
// ---------------------------------------------------------------------------

int32_t setup_device_pool() {
    static uint64_t done_mask = 0;
    int dev = 0;
    PPG_CUDA(cudaGetDevice(&dev));
    if (dev < 64 && (done_mask >> dev) & 1) return PPG_OK;
    cudaMemPool_t pool;
    PPG_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
    uint64_t thr = ~0ull;   // keep freed scratch cached in the pool
    PPG_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
    if (dev < 64) done_mask |= (1ull << dev);
    return PPG_OK;
}

int device_sm_count() {
    static std::atomic<int> cached[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        dev = -1;
    }
    int v = dev >= 0 ? cached[dev].load(std::memory_order_relaxed) : 0;
    if (v == 0) {
        if (dev < 0 || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) !=
                           cudaSuccess || v < 1) {
            cudaGetLastError();
            v = 1;
        }
        if (dev >= 0) cached[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

static int64_t pad_ld(int32_t n) { return ((int64_t)n + 63) / 64 * 64; }

// Pinned host buffer for the per-step status read (one per host thread,
// allocated on first use and kept for the life of the process): 8 doubles
// of GmresState::scal, then the CGS2 error flag at element 8.
static int32_t status_buffer(double** out) {
    static thread_local double* buf = nullptr;
    if (!buf) {
        void* p = nullptr;
        PPG_CUDA(cudaMallocHost(&p, 16 * sizeof(double)));
        buf = (double*)p;
    }
    *out = buf;
    return PPG_OK;
}

int32_t check_csr(const ppg_csr* A, int dtype_required) {
    if (!A || A->n < 1 || A->nnz < 0 || !A->rowptr || (A->nnz > 0 && (!A->colind || !A->vals)))
        return PPG_ERR_ARG;
    if (A->dtype != PPG_F64 && A->dtype != PPG_F32) return PPG_ERR_ARG;
    if (dtype_required >= 0 && A->dtype != dtype_required) return PPG_ERR_ARG;
    return PPG_OK;
}

int32_t check_roots(const ppg_roots* r) {
    if (!r || r->n_total < 1 || !r->re || !r->im) return PPG_ERR_ARG;
    const int d = r->n_total;
    for (int i = 0; i < d;) {
        if (!std::isfinite(r->re[i]) || !std::isfinite(r->im[i])) return PPG_ERR_ARG;
        if (r->im[i] == 0.0) {
            if (r->re[i] == 0.0) return PPG_ERR_ARG;
            i += 1;
        } else {
            if (i + 1 >= d || r->re[i + 1] != r->re[i] || r->im[i + 1] != -r->im[i])
                return PPG_ERR_ARG;
            i += 2;
        }
    }
    return PPG_OK;
}

struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    bool on = false;
    int32_t init(bool enable) {
        on = enable;
        if (!on) return PPG_OK;
        PPG_CUDA(cudaEventCreate(&a));
        PPG_CUDA(cudaEventCreate(&b));
        return PPG_OK;
    }
    void start(cudaStream_t s) { if (on) cudaEventRecord(a, s); }
    void stop(cudaStream_t s) { if (on) cudaEventRecord(b, s); }
    // after the stream was synchronised
    double ms() {
        if (!on) return 0.0;
        float t = 0.f;
        cudaEventElapsedTime(&t, a, b);
        return (double)t;
    }
    ~EventPair() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

// ---------------------------------------------------------------------------
// GMRES core shared by the plain and flexible forms
// ---------------------------------------------------------------------------

struct SolveCore {
    // inputs
    const ppg_csr* A64;
    const ppg_csr* A32;            // flex only
    const ppg_roots* roots;        // may be null (plain GMRES)
    const double* b;
    double* x;
    int m;
    double tol;
    ppg_opts opts;
    bool flex;
    cudaStream_t s;
    // workspace
    double* V = nullptr;
    int64_t ldv = 0;
    float* Z32 = nullptr;
    double* va = nullptr;
    double* vb = nullptr;
    double* vc = nullptr;
    double* u = nullptr;
    float* fa = nullptr;
    float* fb = nullptr;
    float* fc = nullptr;
    float* v32 = nullptr;
    float* zh = nullptr;                    // sweep form: p(A) v_j in the plan's ordering
    const ppg_sweep_plan* sweep = nullptr;  // flexible form through a fused-sweep plan
    double* spart = nullptr;
    OrthoWs ows{};
    GmresState gs{};
    std::vector<Step> phi_plan, p_plan;
    ppg_stats st{};
};

// CGS2 of basis column j + 1 (w) against columns 0..j: h1 = V^T w; w -= V h1;
// h2 = V^T w; w -= V h2 with ||w||^2.  With opts.cgs2_fused the middle two
// passes run as one pass over V when the basis layout allows it.
static int32_t cgs2_column(SolveCore& c, int j, double* w, bool with_self, EventPair* ev) {
    const int32_t n = c.A64->n;
    if (ev) ev->start(c.s);
    PPG_TRY(launch_cgs_dot(c.V, c.ldv, j + 1, w, n, with_self, c.ows.h1, c.ows, c.s));
    if (c.opts.cgs2_fused && cgs_fused_ok(c.V, c.ldv, j + 1, w)) {
        PPG_TRY(launch_cgs_sub_dot(c.V, c.ldv, j + 1, w, n, c.ows.h1, c.ows.h2, c.ows, c.s));
    } else {
        PPG_TRY(launch_cgs_update(c.V, c.ldv, j + 1, w, n, c.ows.h1, false, nullptr, c.ows,
                                  c.s));
        PPG_TRY(launch_cgs_dot(c.V, c.ldv, j + 1, w, n, false, c.ows.h2, c.ows, c.s));
    }
    PPG_TRY(launch_cgs_update(c.V, c.ldv, j + 1, w, n, c.ows.h2, true, c.ows.nrm, c.ows, c.s));
    return PPG_OK;
}

// the error flag of the fused CGS2 pass (a staging wait gave up); `flag`
// is host memory filled by a copy the caller has synchronised
static int32_t ortho_status(const unsigned* flag) {
    return *flag != 0u ? PPG_ERR_TIMEOUT : PPG_OK;
}

// Algorithm 4 step 1 with operator M = A, or M = phi_inner(A) when inner is
// given (the second polynomial of double polynomial preconditioning,
// Section 6): d Arnoldi steps with CGS2 from v0, then the host steps.
static int32_t build_core(const ppg_csr* A, int d, const double* v0, const ppg_opts& o,
                          const ppg_roots* inner, ppg_roots* out, double* Hbar_host,
                          cudaStream_t s) {
    PPG_TRY(setup_device_pool());
    const int32_t n = A->n;
    const int ldh = d + 1;
    SolveCore c{};
    c.A64 = A;
    c.s = s;
    c.opts = o;
    c.ldv = pad_ld(n);
    Arena ar;
    ar.add(&c.V, (size_t)c.ldv * (d + 1));
    const int sg = spmv_grid_blocks(n);
    ar.add(&c.spart, (size_t)sg + 1024);
    c.ows.grid = ortho_grid(n);
    ar.add(&c.ows.part, ortho_part_doubles(c.ows.grid));
    ar.add(&c.ows.counter, 4);
    ar.add(&c.ows.h1, ORTHO_MAXC + 2);
    ar.add(&c.ows.h2, ORTHO_MAXC + 2);
    ar.add(&c.ows.nrm, 4);
    ar.add(&c.gs.Hraw, (size_t)ldh * d);
    ar.add(&c.gs.scal, 8);
    if (inner) {
        ar.add(&c.va, (size_t)n);
        ar.add(&c.vb, (size_t)n);
        ar.add(&c.vc, (size_t)n);
    }
    c.gs.R = nullptr;
    PPG_TRY(ar.alloc(s));
    struct Guard { Arena& a; cudaStream_t s; ~Guard() { a.release(s); } } guard{ar, s};
    PPG_CUDA(cudaMemsetAsync(c.ows.counter, 0, 4 * sizeof(unsigned), s));
    PPG_CUDA(cudaMemsetAsync(c.gs.scal, 0, 8 * sizeof(double), s));
    PPG_CUDA(cudaMemsetAsync(c.gs.Hraw, 0, sizeof(double) * ldh * d, s));
    std::vector<Step> inner_phi;
    if (inner) inner_phi = plan_phi(inner->re, inner->im, inner->n_total, false);
    int nparts = 0;
    PPG_TRY(launch_norm2_part(v0, n, c.spart, s, &nparts));
    PPG_TRY(launch_reduce_norm(c.spart, nparts, c.gs.scal, nullptr, s));
    PPG_TRY(launch_scale(v0, c.V, n, c.gs.scal + 4, s));
    for (int j = 0; j < d; ++j) {
        double* vj = c.V + (size_t)j * c.ldv;
        double* w = c.V + (size_t)(j + 1) * c.ldv;
        if (inner) {
            Buffers b{};
            b.ptr[B_IN] = vj;
            b.ptr[B_OUT] = w;
            b.ptr[B_A] = c.va;
            b.ptr[B_B] = c.vb;
            b.ptr[B_C] = c.vc;
            PPG_TRY(run_plan<double>(inner_phi, A->rowptr, A->colind, (const double*)A->vals, n,
                                     A->nnz, b, s, nullptr));
        } else {
            StepArgs<double> a{};
            a.rowptr = A->rowptr;
            a.colind = A->colind;
            a.vals = (const double*)A->vals;
            a.n = n;
            a.flags = keep_a_flag(a.n, A->nnz, 8, 3);
            a.x = vj;
            a.o0 = w;
            int32_t g = launch_step<double>(OP_SPMV, a, s);
            if (g < 0) return g;
        }
        PPG_TRY(cgs2_column(c, j, w, true, nullptr));
        PPG_TRY(launch_finish_column(c.gs, ldh, j, c.ows.h1, c.ows.h2, c.ows.nrm, false, 1.0,
                                     1e-13, s));
        PPG_TRY(launch_scale(w, w, n, c.gs.scal + 2, s));
    }
    std::vector<double> H((size_t)ldh * d), sc(8);
    PPG_CUDA(cudaMemcpyAsync(H.data(), c.gs.Hraw, sizeof(double) * ldh * d,
                             cudaMemcpyDeviceToHost, s));
    PPG_CUDA(cudaMemcpyAsync(sc.data(), c.gs.scal, sizeof(double) * 8, cudaMemcpyDeviceToHost, s));
    unsigned oflag = 0;
    PPG_CUDA(cudaMemcpyAsync(&oflag, c.ows.counter + 3, sizeof(unsigned), cudaMemcpyDeviceToHost,
                             s));
    PPG_CUDA(cudaStreamSynchronize(s));
    PPG_TRY(ortho_status(&oflag));
    if (Hbar_host) std::memcpy(Hbar_host, H.data(), sizeof(double) * ldh * d);
    if (!std::isfinite(sc[3]) || sc[3] == 0.0) return PPG_ERR_ARG;   // v0 zero or non-finite
    const bool brk = sc[5] != 0.0;
    const int d_eff = brk ? (int)sc[6] + 1 : d;
    int32_t rc = ppg_roots_from_hessenberg(H.data(), ldh, d_eff, &o, out);
    if (rc != PPG_OK) return rc;
    return brk ? PPG_LUCKY_BREAKDOWN : PPG_OK;
}

static int32_t run_solve(SolveCore& c) {
    const int32_t n = c.A64->n;
    const int64_t nnz = c.A64->nnz;
    const int m = c.m;
    const int ldh = m + 1;
    cudaStream_t s = c.s;
    const bool pp = c.roots && c.roots->n_total > 0;
    const int d = pp ? c.roots->n_total : 1;
    const int64_t launches0 = g_launches;
    PPG_TRY(setup_device_pool());

    if (pp) {
        c.phi_plan = plan_phi(c.roots->re, c.roots->im, d, false);
        // plain form: x += p(A) u accumulates into x; flexible form: z_j =
        // p(A) v_j starts from zero
        c.p_plan = plan_p(c.roots->re, c.roots->im, d, !c.flex);
    }
    Arena ar;
    c.ldv = pad_ld(n);
    ar.add(&c.V, (size_t)c.ldv * (m + 1));
    if (c.flex) {
        ar.add(&c.Z32, (size_t)c.ldv * m);
        ar.add(&c.fa, (size_t)n);
        ar.add(&c.fb, (size_t)n);
        ar.add(&c.fc, (size_t)n);
        ar.add(&c.v32, (size_t)n);
        if (c.sweep) ar.add(&c.zh, (size_t)n);
    }
    ar.add(&c.va, (size_t)n);
    ar.add(&c.vb, (size_t)n);
    ar.add(&c.vc, (size_t)n);
    ar.add(&c.u, (size_t)n);
    const int sgrid = spmv_grid_blocks(n);
    ar.add(&c.spart, (size_t)sgrid + 1024);
    c.ows.grid = ortho_grid(n);
    ar.add(&c.ows.part, ortho_part_doubles(c.ows.grid));
    ar.add(&c.ows.counter, 4);
    ar.add(&c.ows.h1, ORTHO_MAXC + 2);
    ar.add(&c.ows.h2, ORTHO_MAXC + 2);
    ar.add(&c.ows.nrm, 4);
    ar.add(&c.gs.R, (size_t)ldh * m);
    ar.add(&c.gs.cs, (size_t)m);
    ar.add(&c.gs.sn, (size_t)m);
    ar.add(&c.gs.g, (size_t)m + 1);
    ar.add(&c.gs.y, (size_t)m);
    ar.add(&c.gs.scal, 8);
    c.gs.Hraw = nullptr;
    PPG_TRY(ar.alloc(s));
    struct Guard { Arena& a; cudaStream_t s; ~Guard() { a.release(s); } } guard{ar, s};

    PPG_CUDA(cudaMemsetAsync(c.ows.counter, 0, 4 * sizeof(unsigned), s));
    PPG_CUDA(cudaMemsetAsync(c.gs.scal, 0, 8 * sizeof(double), s));

    // timers of two consecutive Arnoldi steps (the look-ahead records the
    // next step's before the current one is read) and of the restart update
    EventPair ev_poly[2], ev_orth[2], ev_restart;
    for (int i = 0; i < 2; ++i) {
        PPG_TRY(ev_poly[i].init(c.opts.timing != 0));
        PPG_TRY(ev_orth[i].init(c.opts.timing != 0));
    }
    PPG_TRY(ev_restart.init(c.opts.timing != 0));
    // marks the copy of a step's residual estimate: the host waits for it,
    // not for the look-ahead enqueued behind it
    struct ReadyEvent {
        cudaEvent_t e = nullptr;
        ~ReadyEvent() { if (e) cudaEventDestroy(e); }
    } ready;
    PPG_CUDA(cudaEventCreateWithFlags(&ready.e, cudaEventDisableTiming));
    cudaEvent_t ev_ready = ready.e;

    c.st = ppg_stats{};
    double* scal_h = nullptr;
    PPG_TRY(status_buffer(&scal_h));
    int nparts = 0;

    // ||b||
    PPG_TRY(launch_norm2_part(c.b, n, c.spart, s, &nparts));
    PPG_TRY(launch_reduce_norm(c.spart, nparts, c.gs.scal, nullptr, s));
    PPG_CUDA(cudaMemcpyAsync(scal_h, c.gs.scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
    PPG_CUDA(cudaStreamSynchronize(s));
    const double bnorm = scal_h[3];
    c.st.dots += 1;
    if (!std::isfinite(bnorm)) return PPG_ERR_NONFINITE;
    if (bnorm == 0.0) {
        PPG_TRY(launch_fill(c.x, 0.0, n, s));
        PPG_CUDA(cudaStreamSynchronize(s));
        c.st.converged = 1;
        c.st.true_relres = 0.0;
        c.st.launches = g_launches - launches0;
        return PPG_OK;
    }

    // initial residual into V[:, 0]
    double beta;
    {
        StepArgs<double> a{};
        a.rowptr = c.A64->rowptr;
        a.colind = c.A64->colind;
        a.vals = (const double*)c.A64->vals;
        a.n = n;
        a.flags = keep_a_flag(a.n, c.A64->nnz, 8, 3);
        if (c.opts.x0_given) {
            a.x = c.x;
            a.a0 = c.b;
            a.o0 = c.V;
            a.part = c.spart;
            int32_t g = launch_step<double>(OP_RESID, a, s);
            if (g < 0) return g;
            PPG_TRY(launch_reduce_norm(c.spart, g, c.gs.scal, c.gs.g, s));
            c.st.mvps += 1;
            c.st.dots += 1;
        } else {
            PPG_TRY(launch_fill(c.x, 0.0, n, s));
            PPG_CUDA(cudaMemcpyAsync(c.V, c.b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
            PPG_TRY(launch_reduce_norm(c.spart, nparts, c.gs.scal, c.gs.g, s));
        }
        PPG_CUDA(cudaMemcpyAsync(scal_h, c.gs.scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
        PPG_CUDA(cudaStreamSynchronize(s));
        beta = scal_h[3];
    }
    c.st.true_relres = beta / bnorm;
    if (!std::isfinite(beta)) return PPG_ERR_NONFINITE;
    bool converged = c.st.true_relres <= c.tol;

    Buffers phib{};
    phib.ptr[B_A] = c.va;
    phib.ptr[B_B] = c.vb;
    phib.ptr[B_C] = c.vc;
    Buffers pb{};

    // One Arnoldi step: the operator chain (phi(A) v_j by Algorithm 1; in the
    // flexible form z_j = p(A) v_j by Algorithm 3 in FP32 and w = A z_j; plain
    // GMRES: w = A v_j), CGS2, the Givens update, and the copy of the
    // residual estimate to the host.
    //
    // Look-ahead: before the host waits for step j's estimate, the scaling of
    // v_{j+1} and the first `nahead` chain kernels of step j + 1 are already
    // enqueued, so the GPU stays busy across the host round trip.  If the
    // cycle stops at step j they have written only work vectors (the prefix
    // never includes a chain's last step) and basis column j + 1, which the
    // update does not read.
    constexpr int kLookahead = 2;
    const std::vector<Step>* chain = pp ? (c.flex ? &c.p_plan : &c.phi_plan) : nullptr;
    // (the fused-sweep chain runs whole: its pairs must not be split)
    const int nahead = (chain && !c.sweep)
                           ? std::max(0, std::min(kLookahead, (int)chain->size() - 1))
                           : 0;
    auto chain_steps = [&](int j, int i0, int i1, double* by) -> int32_t {
        if (c.sweep) {
            Buffers fb{};
            fb.ptr[B_IN] = c.v32;
            fb.ptr[B_P] = c.zh;
            fb.ptr[B_A] = c.fa;
            fb.ptr[B_B] = c.fb;
            fb.ptr[B_C] = c.fc;
            if (i0 != 0 || i1 != (int)c.p_plan.size()) return PPG_ERR_ARG;
            PPG_TRY(sweep_run_chain(c.sweep, c.p_plan, fb, s));
            if (by) *by = sweep_chain_bytes(c.sweep, c.p_plan);
            return sweep_scatter(c.sweep, c.zh, c.Z32 + (size_t)j * c.ldv, s);
        }
        if (c.flex) {
            Buffers fb{};
            fb.ptr[B_IN] = c.v32;
            fb.ptr[B_P] = c.Z32 + (size_t)j * c.ldv;
            fb.ptr[B_A] = c.fa;
            fb.ptr[B_B] = c.fb;
            fb.ptr[B_C] = c.fc;
            return run_steps<float>(c.p_plan, i0, i1, c.A32->rowptr, c.A32->colind,
                                    (const float*)c.A32->vals, n, nnz, fb, s, by);
        }
        phib.ptr[B_IN] = c.V + (size_t)j * c.ldv;
        phib.ptr[B_OUT] = c.V + (size_t)(j + 1) * c.ldv;
        return run_steps<double>(c.phi_plan, i0, i1, c.A64->rowptr, c.A64->colind,
                                 (const double*)c.A64->vals, n, nnz, phib, s, by);
    };
    // start of step j: the FP32 cast of v_j (flexible form), the chain timer
    // (root steps only, not the cast) and chain steps [0, upto)
    auto begin_step = [&](int j, int e, int upto, double* by) -> int32_t {
        *by = 0.0;
        if (c.sweep) {
            PPG_TRY(sweep_gather(c.sweep, c.V + (size_t)j * c.ldv, true, c.v32, s));
        } else if (c.flex) {
            PPG_TRY(launch_cast_f64_f32(c.V + (size_t)j * c.ldv, c.v32, n, s));
        }
        ev_poly[e].start(s);
        if (chain && upto > 0) PPG_TRY(chain_steps(j, 0, upto, by));
        return PPG_OK;
    };
    // the rest of step j from chain step `from` on
    auto finish_step = [&](int j, int e, int from, double* by) -> int32_t {
        double* vj = c.V + (size_t)j * c.ldv;
        double* w = c.V + (size_t)(j + 1) * c.ldv;
        StepArgs<double> a{};
        a.rowptr = c.A64->rowptr;
        a.colind = c.A64->colind;
        a.vals = (const double*)c.A64->vals;
        a.n = n;
        a.flags = keep_a_flag(a.n, c.A64->nnz, 8, 3);
        a.o0 = w;
        if (c.flex) {
            float* zj = c.Z32 + (size_t)j * c.ldv;
            if (pp) {
                double b2 = 0;
                PPG_TRY(chain_steps(j, from, (int)chain->size(), &b2));
                *by += b2;
            } else {
                PPG_CUDA(cudaMemcpyAsync(zj, c.v32, sizeof(float) * n, cudaMemcpyDeviceToDevice,
                                         s));
            }
            ev_poly[e].stop(s);
            PPG_TRY(launch_cast_f32_f64(zj, c.u, n, s));
            a.x = c.u;
            const int32_t g = launch_step<double>(OP_SPMV, a, s);
            if (g < 0) return g;
        } else if (pp) {
            double b2 = 0;
            PPG_TRY(chain_steps(j, from, (int)chain->size(), &b2));
            *by += b2;
            ev_poly[e].stop(s);
        } else {
            a.x = vj;
            const int32_t g = launch_step<double>(OP_SPMV, a, s);
            if (g < 0) return g;
            ev_poly[e].stop(s);
            *by = step_bytes(OP_SPMV, 0, n, nnz, 8);
        }
        PPG_TRY(cgs2_column(c, j, w, false, &ev_orth[e]));
        PPG_TRY(launch_finish_column(c.gs, ldh, j, c.ows.h1, c.ows.h2, c.ows.nrm, true, bnorm,
                                     0.0, s));
        ev_orth[e].stop(s);
        PPG_CUDA(cudaMemcpyAsync(scal_h, c.gs.scal, 4 * sizeof(double), cudaMemcpyDeviceToHost,
                                 s));
        return PPG_OK;
    };

    const int max_cycles = c.opts.max_cycles > 0 ? c.opts.max_cycles : 10000;
    for (int cyc = 0; cyc < max_cycles && !converged; ++cyc) {
        c.st.cycles += 1;
        PPG_TRY(launch_scale(c.V, c.V, n, c.gs.scal + 4, s));
        int k = 0;
        int from = 0;        // chain steps of step j already enqueued
        double by_cur = 0;   // their algorithmic bytes
        PPG_TRY(begin_step(0, 0, 0, &by_cur));
        for (int j = 0; j < m; ++j) {
            const int e = j & 1;
            double* w = c.V + (size_t)(j + 1) * c.ldv;
            PPG_TRY(finish_step(j, e, from, &by_cur));
            PPG_CUDA(cudaEventRecord(ev_ready, s));
            const double by_step = by_cur;
            from = 0;
            if (j + 1 < m) {   // look-ahead into step j + 1
                PPG_TRY(launch_scale(w, w, n, c.gs.scal + 2, s));
                PPG_TRY(begin_step(j + 1, e ^ 1, nahead, &by_cur));
                from = nahead;
            }
            PPG_CUDA(cudaEventSynchronize(ev_ready));
            c.st.poly_ms += ev_poly[e].ms();
            c.st.ortho_ms += ev_orth[e].ms();
            c.st.poly_bytes += by_step;
            c.st.poly_launches += chain ? (c.sweep ? sweep_chain_launches(c.sweep, *chain)
                                                   : (int64_t)chain->size())
                                        : (c.flex ? 0 : 1);
            c.st.mvps += pp ? d : 1;   // flexible form: d-1 in p(A) v_j, one for A z_j
            c.st.iters += 1;
            c.st.dots += 2 * (j + 1) + 1;
            k = j + 1;
            const double est = scal_h[0];
            const double hn = scal_h[1];
            c.st.est_relres = est;
            if (!std::isfinite(est) || !std::isfinite(hn)) return PPG_ERR_NONFINITE;
            if (est <= c.tol || hn == 0.0) break;
        }
        PPG_TRY(launch_backsolve(c.gs, ldh, k, s));
        if (c.flex) {
            PPG_TRY(launch_gemv_acc<float>(c.Z32, c.ldv, k, c.gs.y, c.x, n, true, s));
        } else if (pp) {
            PPG_TRY(launch_gemv_acc<double>(c.V, c.ldv, k, c.gs.y, c.u, n, false, s));
            pb.ptr[B_IN] = c.u;
            pb.ptr[B_P] = c.x;
            pb.ptr[B_A] = c.va;
            pb.ptr[B_B] = c.vb;
            pb.ptr[B_C] = c.vc;
            double by = 0;
            ev_restart.start(s);
            PPG_TRY(run_plan<double>(c.p_plan, c.A64->rowptr, c.A64->colind,
                                     (const double*)c.A64->vals, n, nnz, pb, s, &by));
            ev_restart.stop(s);
            c.st.poly_bytes += by;
            c.st.poly_launches += (int64_t)c.p_plan.size();
            c.st.mvps += d - 1;
        } else {
            PPG_TRY(launch_gemv_acc<double>(c.V, c.ldv, k, c.gs.y, c.x, n, true, s));
        }
        // true residual r = b - A x into V[:, 0]
        StepArgs<double> a{};
        a.rowptr = c.A64->rowptr;
        a.colind = c.A64->colind;
        a.vals = (const double*)c.A64->vals;
        a.n = n;
        a.flags = keep_a_flag(a.n, c.A64->nnz, 8, 3);
        a.x = c.x;
        a.a0 = c.b;
        a.o0 = c.V;
        a.part = c.spart;
        int32_t g = launch_step<double>(OP_RESID, a, s);
        if (g < 0) return g;
        PPG_TRY(launch_reduce_norm(c.spart, g, c.gs.scal, c.gs.g, s));
        c.st.mvps += 1;
        c.st.dots += 1;
        PPG_CUDA(cudaMemcpyAsync(scal_h, c.gs.scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
        PPG_CUDA(cudaMemcpyAsync(scal_h + 8, c.ows.counter + 3, sizeof(unsigned),
                                 cudaMemcpyDeviceToHost, s));
        PPG_CUDA(cudaStreamSynchronize(s));
        PPG_TRY(ortho_status(reinterpret_cast<const unsigned*>(scal_h + 8)));
        if (pp && !c.flex) c.st.poly_ms += ev_restart.ms();
        beta = scal_h[3];
        if (!std::isfinite(beta)) return PPG_ERR_NONFINITE;
        c.st.true_relres = beta / bnorm;
        converged = c.st.true_relres <= c.tol;
    }
    c.st.converged = converged ? 1 : 0;
    c.st.launches = g_launches - launches0;
    return converged ? PPG_OK : PPG_NOT_CONVERGED;
}

// Restarted GMRES(m) on a polynomial of an operator M, for the two
// variants of Sections 5.2 and 6:
//  * double polynomial (inner != NULL): M = phi_1(A) with phi_1 from the
//    inner roots; the solve runs GMRES on phi_2(M) z = b with phi_2 from
//    c.roots, accumulates x' = p_2(M) z over the restarts (each restart from
//    the true residual b - M x'), and returns x = p_1(A) x';
//  * changing polynomial (rebuild_d > 0): M = A, and the polynomial is
//    rebuilt by GMRES(rebuild_d) from the current residual at the start of
//    every cycle.
// Operator products of a composite M run its Algorithm 1 chain into a work
// vector, and the outer root step is then applied elementwise.
static int32_t run_solve_ext(SolveCore& c, const ppg_roots* inner, int rebuild_d) {
    const int32_t n = c.A64->n;
    const int64_t nnz = c.A64->nnz;
    const int m = c.m;
    const int ldh = m + 1;
    cudaStream_t s = c.s;
    const ppg_csr* A = c.A64;
    const double* vals = (const double*)A->vals;
    const int64_t launches0 = g_launches;
    PPG_TRY(setup_device_pool());
    const int dM = inner ? inner->n_total : 1;
    std::vector<Step> inner_phi;
    if (inner) inner_phi = plan_phi(inner->re, inner->im, inner->n_total, false);

    Arena ar;
    c.ldv = pad_ld(n);
    double *ia = nullptr, *ib = nullptr, *ic = nullptr, *S = nullptr, *xp = nullptr;
    ar.add(&c.V, (size_t)c.ldv * (m + 1));
    ar.add(&c.va, (size_t)n);
    ar.add(&c.vb, (size_t)n);
    ar.add(&c.vc, (size_t)n);
    ar.add(&c.u, (size_t)n);
    ar.add(&ia, (size_t)n);
    ar.add(&ib, (size_t)n);
    ar.add(&ic, (size_t)n);
    ar.add(&S, (size_t)n);
    ar.add(&xp, (size_t)n);
    const int sgrid = spmv_grid_blocks(n);
    ar.add(&c.spart, (size_t)sgrid + 1024);
    c.ows.grid = ortho_grid(n);
    ar.add(&c.ows.part, ortho_part_doubles(c.ows.grid));
    ar.add(&c.ows.counter, 4);
    ar.add(&c.ows.h1, ORTHO_MAXC + 2);
    ar.add(&c.ows.h2, ORTHO_MAXC + 2);
    ar.add(&c.ows.nrm, 4);
    ar.add(&c.gs.R, (size_t)ldh * m);
    ar.add(&c.gs.cs, (size_t)m);
    ar.add(&c.gs.sn, (size_t)m);
    ar.add(&c.gs.g, (size_t)m + 1);
    ar.add(&c.gs.y, (size_t)m);
    ar.add(&c.gs.scal, 8);
    c.gs.Hraw = nullptr;
    PPG_TRY(ar.alloc(s));
    struct Guard { Arena& a; cudaStream_t s; ~Guard() { a.release(s); } } guard{ar, s};
    PPG_CUDA(cudaMemsetAsync(c.ows.counter, 0, 4 * sizeof(unsigned), s));
    PPG_CUDA(cudaMemsetAsync(c.gs.scal, 0, 8 * sizeof(double), s));

    // y = M x
    auto apply_M = [&](const double* xin, double* yout) -> int32_t {
        if (inner) {
            Buffers b{};
            b.ptr[B_IN] = const_cast<double*>(xin);
            b.ptr[B_OUT] = yout;
            b.ptr[B_A] = ia;
            b.ptr[B_B] = ib;
            b.ptr[B_C] = ic;
            return run_plan<double>(inner_phi, A->rowptr, A->colind, vals, n, nnz, b, s, nullptr);
        }
        StepArgs<double> a{};
        a.rowptr = A->rowptr;
        a.colind = A->colind;
        a.vals = vals;
        a.n = n;
        a.flags = keep_a_flag(n, nnz, 8, 3);
        a.x = xin;
        a.o0 = yout;
        const int32_t g = launch_step<double>(OP_SPMV, a, s);
        return g < 0 ? g : PPG_OK;
    };
    // one polynomial of M (a plan built for a single SpMV per product)
    auto run_outer = [&](const std::vector<Step>& plan, const Buffers& bufs) -> int32_t {
        if (!inner)
            return run_plan<double>(plan, A->rowptr, A->colind, vals, n, nnz, bufs, s, nullptr);
        for (const Step& st : plan) {
            double* X = (double*)bufs.ptr[st.x];
            if (st.op == -1) {   // degree one: P = c1 v (+ P), no product
                const bool pz = st.flags & F_PZERO;
                PPG_TRY(launch_axpby<double>(st.c1, X, pz ? 0.0 : 1.0,
                                             pz ? nullptr : (double*)bufs.ptr[B_P],
                                             (double*)bufs.ptr[B_P], n, s));
                continue;
            }
            if (st.op == OP_SPMV) {
                PPG_TRY(apply_M(X, (double*)bufs.ptr[st.o0]));
                continue;
            }
            PPG_TRY(apply_M(X, S));
            StepArgs<double> a{};
            a.n = n;
            a.a0 = st.a0 >= 0 ? (const double*)bufs.ptr[st.a0] : nullptr;
            a.a1 = st.a1 >= 0 ? (const double*)bufs.ptr[st.a1] : nullptr;
            a.a2 = st.a2 >= 0 ? (const double*)bufs.ptr[st.a2] : nullptr;
            a.o0 = st.o0 >= 0 ? (double*)bufs.ptr[st.o0] : nullptr;
            a.o1 = st.o1 >= 0 ? (double*)bufs.ptr[st.o1] : nullptr;
            a.c1 = st.c1;
            a.c2 = st.c2;
            a.c3 = st.c3;
            a.flags = st.flags;
            const int32_t g = launch_ew_step<double>(st.op, a, S, s);
            if (g < 0) return g;
        }
        return PPG_OK;
    };

    c.st = ppg_stats{};
    double* scal_h = nullptr;
    PPG_TRY(status_buffer(&scal_h));
    int nparts = 0;
    PPG_TRY(launch_norm2_part(c.b, n, c.spart, s, &nparts));
    PPG_TRY(launch_reduce_norm(c.spart, nparts, c.gs.scal, c.gs.g, s));
    PPG_CUDA(cudaMemcpyAsync(scal_h, c.gs.scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
    PPG_CUDA(cudaStreamSynchronize(s));
    const double bnorm = scal_h[3];
    c.st.dots += 1;
    if (!std::isfinite(bnorm)) return PPG_ERR_NONFINITE;
    double* xs = inner ? xp : c.x;   // the iterate of the outer solve
    PPG_TRY(launch_fill(xs, 0.0, n, s));
    if (bnorm == 0.0) {
        PPG_TRY(launch_fill(c.x, 0.0, n, s));
        PPG_CUDA(cudaStreamSynchronize(s));
        c.st.converged = 1;
        c.st.true_relres = 0.0;
        c.st.launches = g_launches - launches0;
        return PPG_OK;
    }
    PPG_CUDA(cudaMemcpyAsync(c.V, c.b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    double beta = bnorm;
    c.st.true_relres = 1.0;
    bool converged = false;

    // the outer polynomial (rebuilt every cycle in the changing form)
    std::vector<double> rre, rim;
    ppg_roots rr{};
    const ppg_roots* outer = c.roots;
    Buffers pb{}, phib{};
    phib.ptr[B_A] = c.va;
    phib.ptr[B_B] = c.vb;
    phib.ptr[B_C] = c.vc;
    std::vector<Step> phi_plan, p_plan;
    if (!rebuild_d) {
        phi_plan = plan_phi(outer->re, outer->im, outer->n_total, false);
        p_plan = plan_p(outer->re, outer->im, outer->n_total, true);
    }
    const int max_cycles = c.opts.max_cycles > 0 ? c.opts.max_cycles : 10000;
    for (int cyc = 0; cyc < max_cycles && !converged; ++cyc) {
        c.st.cycles += 1;
        if (rebuild_d) {
            // Section 5.2: GMRES(rebuild_d) from the current residual r (in V_0)
            const int cap = 4 * rebuild_d + 8;
            rre.assign(cap, 0.0);
            rim.assign(cap, 0.0);
            rr = ppg_roots{0, 0, 0, cap, rre.data(), rim.data(), nullptr};
            const int32_t rc = build_core(A, rebuild_d, c.V, c.opts, nullptr, &rr, nullptr, s);
            if (rc < 0) return rc;
            outer = &rr;
            phi_plan = plan_phi(rr.re, rr.im, rr.n_total, false);
            p_plan = plan_p(rr.re, rr.im, rr.n_total, true);
            c.st.mvps += rebuild_d;
        }
        const int d = outer->n_total;
        PPG_TRY(launch_scale(c.V, c.V, n, c.gs.scal + 4, s));
        int k = 0;
        for (int j = 0; j < m; ++j) {
            double* vj = c.V + (size_t)j * c.ldv;
            double* w = c.V + (size_t)(j + 1) * c.ldv;
            phib.ptr[B_IN] = vj;
            phib.ptr[B_OUT] = w;
            PPG_TRY(run_outer(phi_plan, phib));
            c.st.mvps += (int64_t)d * dM;
            PPG_TRY(cgs2_column(c, j, w, false, nullptr));
            PPG_TRY(launch_finish_column(c.gs, ldh, j, c.ows.h1, c.ows.h2, c.ows.nrm, true,
                                         bnorm, 0.0, s));
            PPG_CUDA(cudaMemcpyAsync(scal_h, c.gs.scal, 4 * sizeof(double),
                                     cudaMemcpyDeviceToHost, s));
            PPG_CUDA(cudaStreamSynchronize(s));
            c.st.iters += 1;
            c.st.dots += 2 * (j + 1) + 1;
            k = j + 1;
            const double est = scal_h[0], hn = scal_h[1];
            c.st.est_relres = est;
            if (!std::isfinite(est) || !std::isfinite(hn)) return PPG_ERR_NONFINITE;
            if (est <= c.tol || hn == 0.0) break;
            if (j + 1 < m) PPG_TRY(launch_scale(w, w, n, c.gs.scal + 2, s));
        }
        PPG_TRY(launch_backsolve(c.gs, ldh, k, s));
        PPG_TRY(launch_gemv_acc<double>(c.V, c.ldv, k, c.gs.y, c.u, n, false, s));
        pb.ptr[B_IN] = c.u;
        pb.ptr[B_P] = xs;
        pb.ptr[B_A] = c.va;
        pb.ptr[B_B] = c.vb;
        pb.ptr[B_C] = c.vc;
        PPG_TRY(run_outer(p_plan, pb));
        c.st.mvps += (int64_t)(d - 1) * dM;
        // true residual r = b - M x' into V_0
        PPG_TRY(apply_M(xs, S));
        StepArgs<double> a{};
        a.n = n;
        a.a0 = c.b;
        a.o0 = c.V;
        a.part = c.spart;
        const int32_t g = launch_ew_step<double>(OP_RESID, a, S, s);
        if (g < 0) return g;
        PPG_TRY(launch_reduce_norm(c.spart, g, c.gs.scal, c.gs.g, s));
        c.st.mvps += dM;
        c.st.dots += 1;
        PPG_CUDA(cudaMemcpyAsync(scal_h, c.gs.scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
        PPG_CUDA(cudaMemcpyAsync(scal_h + 8, c.ows.counter + 3, sizeof(unsigned),
                                 cudaMemcpyDeviceToHost, s));
        PPG_CUDA(cudaStreamSynchronize(s));
        PPG_TRY(ortho_status(reinterpret_cast<const unsigned*>(scal_h + 8)));
        beta = scal_h[3];
        if (!std::isfinite(beta)) return PPG_ERR_NONFINITE;
        c.st.true_relres = beta / bnorm;
        converged = c.st.true_relres <= c.tol;
    }
    if (inner) {
        // x = p_1(A) x'
        Buffers b{};
        b.ptr[B_IN] = xp;
        b.ptr[B_P] = c.x;
        b.ptr[B_A] = ia;
        b.ptr[B_B] = ib;
        b.ptr[B_C] = ic;
        PPG_TRY(run_plan<double>(plan_p(inner->re, inner->im, inner->n_total, false), A->rowptr,
                                 A->colind, vals, n, nnz, b, s, nullptr));
        c.st.mvps += dM - 1;
        PPG_CUDA(cudaStreamSynchronize(s));
    }
    c.st.converged = converged ? 1 : 0;
    c.st.launches = g_launches - launches0;
    return converged ? PPG_OK : PPG_NOT_CONVERGED;
}

}  // namespace ppg

using namespace ppg;

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

int32_t ppg_abi_version(void) { return PPG_ABI_VERSION; }

const char* ppg_strerror(int32_t code) {
    switch (code) {
        case PPG_OK: return "ok";
        case PPG_NOT_CONVERGED: return "not converged within max_cycles";
        case PPG_LUCKY_BREAKDOWN: return "Arnoldi breakdown: invariant Krylov subspace";
        case PPG_ERR_ARG: return "invalid argument";
        case PPG_ERR_CSR: return "invalid CSR structure";
        case PPG_ERR_SINGULAR_H: return "H_dd is singular";
        case PPG_ERR_NONFINITE: return "non-finite value encountered";
        case PPG_ERR_CUDA: return "CUDA runtime error";
        case PPG_ERR_CAPACITY: return "roots capacity too small";
        case PPG_ERR_EIG: return "Hessenberg QR did not converge";
        case PPG_ERR_NOMEM: return "device scratch allocation failed";
        case PPG_ERR_TOO_LARGE: return "n exceeds PPG_NOALLOC_MAX_N (1048576), the fixed work area of ppg_apply_poly_noalloc";
        case PPG_ERR_TIMEOUT: return "a bounded wait inside a kernel gave up (staging or grid barrier did not complete)";
        default: return "unknown status";
    }
}

const char* ppg_last_cuda_error(void) { return g_cuda_err; }

int64_t ppg_launch_count(void) { return g_launches; }

void ppg_default_opts(ppg_opts* o) {
    if (!o) return;
    o->max_cycles = 10000;
    o->stability_control = 1;
    o->pof_threshold_log10 = 4.0;
    o->pof_step_log10 = 14.0;
    o->timing = 0;
    o->x0_given = 0;
    o->batch_mode = 0;
    o->cgs2_fused = 0;
    o->wait_timeout_ms = 5000.0;
}

int32_t ppg_harmonic_ritz(const double* Hbar, int32_t ldh, int32_t d, double* re, double* im) {
    return host_harmonic_ritz(Hbar, ldh, d, re, im);
}

int32_t ppg_leja_order(int32_t k, const double* re, const double* im, double* ro, double* io) {
    return host_leja(k, re, im, ro, io);
}

int32_t ppg_add_roots(int32_t k, const double* re, const double* im, double thr, double step,
                      ppg_roots* out) {
    return host_add_roots(k, re, im, thr, step, out);
}

int32_t ppg_roots_from_hessenberg(const double* Hbar, int32_t ldh, int32_t d,
                                  const ppg_opts* opts, ppg_roots* out) {
    if (!out || d < 1) return PPG_ERR_ARG;
    ppg_opts o;
    ppg_default_opts(&o);
    if (opts) o = *opts;
    std::vector<double> re(d), im(d), lr(d), li(d);
    int32_t rc = host_harmonic_ritz(Hbar, ldh, d, re.data(), im.data());
    if (rc != PPG_OK) return rc;
    rc = host_leja(d, re.data(), im.data(), lr.data(), li.data());
    if (rc != PPG_OK) return rc;
    if (o.stability_control) {
        return host_add_roots(d, lr.data(), li.data(), o.pof_threshold_log10, o.pof_step_log10,
                              out);
    }
    // no root adding: report pof anyway (huge thresholds add nothing)
    return host_add_roots(d, lr.data(), li.data(), 1e300, 1.0, out);
}

int32_t ppg_csr_validate_host(int32_t n, int32_t nnz, const int32_t* rowptr,
                              const int32_t* colind) {
    if (n < 1 || nnz < 0 || !rowptr || (nnz > 0 && !colind)) return PPG_ERR_ARG;
    if (rowptr[0] != 0 || rowptr[n] != nnz) return PPG_ERR_CSR;
    for (int32_t i = 0; i < n; ++i) {
        if (rowptr[i + 1] < rowptr[i]) return PPG_ERR_CSR;
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            if (colind[k] < 0 || colind[k] >= n) return PPG_ERR_CSR;
            if (k > rowptr[i] && colind[k] <= colind[k - 1]) return PPG_ERR_CSR;
        }
    }
    return PPG_OK;
}

int32_t ppg_spmv(const ppg_csr* A, const void* x, void* y, void* stream) {
    PPG_TRY(check_csr(A, -1));
    if (!x || !y || x == y) return PPG_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (A->dtype == PPG_F64) {
        StepArgs<double> a{};
        a.rowptr = A->rowptr; a.colind = A->colind; a.vals = (const double*)A->vals; a.n = A->n;
        a.x = (const double*)x; a.o0 = (double*)y;
        a.flags = keep_a_flag(A->n, A->nnz, 8, 2);
        int32_t g = launch_step<double>(OP_SPMV, a, s);
        return g < 0 ? g : PPG_OK;
    }
    StepArgs<float> a{};
    a.rowptr = A->rowptr; a.colind = A->colind; a.vals = (const float*)A->vals; a.n = A->n;
    a.x = (const float*)x; a.o0 = (float*)y;
    a.flags = keep_a_flag(A->n, A->nnz, 4, 2);
    int32_t g = launch_step<float>(OP_SPMV, a, s);
    return g < 0 ? g : PPG_OK;
}

static int32_t apply_common(const ppg_csr* A, const ppg_roots* r, const void* v, void* y,
                            void* stream, bool phi) {
    PPG_TRY(check_csr(A, -1));
    PPG_TRY(check_roots(r));
    if (!v || !y || v == y) return PPG_ERR_ARG;
    PPG_TRY(setup_device_pool());
    cudaStream_t s = (cudaStream_t)stream;
    const int d = r->n_total;
    std::vector<Step> plan = phi ? plan_phi(r->re, r->im, d, false)
                                 : plan_p(r->re, r->im, d, false);
    const size_t es = A->dtype == PPG_F64 ? 8 : 4;
    Arena ar;
    char *ba = nullptr, *bb = nullptr, *bc = nullptr;
    ar.add(&ba, es * A->n);
    ar.add(&bb, es * A->n);
    ar.add(&bc, es * A->n);
    PPG_TRY(ar.alloc(s));
    Buffers bufs{};
    bufs.ptr[B_IN] = const_cast<void*>(v);
    bufs.ptr[B_OUT] = y;
    bufs.ptr[B_P] = y;
    bufs.ptr[B_A] = ba;
    bufs.ptr[B_B] = bb;
    bufs.ptr[B_C] = bc;
    int32_t rc;
    if (A->dtype == PPG_F64)
        rc = run_plan<double>(plan, A->rowptr, A->colind, (const double*)A->vals, A->n, A->nnz,
                              bufs, s, nullptr);
    else
        rc = run_plan<float>(plan, A->rowptr, A->colind, (const float*)A->vals, A->n, A->nnz,
                             bufs, s, nullptr);
    ar.release(s);
    return rc;
}

int32_t ppg_apply_poly(const ppg_csr* A, const ppg_roots* r, const void* v, void* y,
                       void* stream) {
    return apply_common(A, r, v, y, stream, false);
}

int32_t ppg_apply_phi(const ppg_csr* A, const ppg_roots* r, const void* v, void* y,
                      void* stream) {
    return apply_common(A, r, v, y, stream, true);
}

int32_t ppg_build_poly(const ppg_csr* A, int32_t d, const double* v0, const ppg_opts* opts,
                       ppg_roots* out, double* Hbar_host, void* stream) {
    PPG_TRY(check_csr(A, PPG_F64));
    if (!v0 || !out || d < 1 || d + 1 > ORTHO_MAXC) return PPG_ERR_ARG;
    ppg_opts o;
    ppg_default_opts(&o);
    if (opts) o = *opts;
    return build_core(A, d, v0, o, nullptr, out, Hbar_host, (cudaStream_t)stream);
}

int32_t ppg_build_poly_composite(const ppg_csr* A, const ppg_roots* inner, int32_t d,
                                 const double* v0, const ppg_opts* opts, ppg_roots* out,
                                 double* Hbar_host, void* stream) {
    PPG_TRY(check_csr(A, PPG_F64));
    if (!v0 || !out || d < 1 || d + 1 > ORTHO_MAXC) return PPG_ERR_ARG;
    if (inner) PPG_TRY(check_roots(inner));
    ppg_opts o;
    ppg_default_opts(&o);
    if (opts) o = *opts;
    return build_core(A, d, v0, o, inner, out, Hbar_host, (cudaStream_t)stream);
}

int32_t ppg_solve(const ppg_csr* A, const ppg_roots* r, const double* b, double* x, int32_t m,
                  double tol, const ppg_opts* opts, ppg_stats* stats, void* stream) {
    PPG_TRY(check_csr(A, PPG_F64));
    if (!b || !x || b == x || m < 1 || m + 1 > ORTHO_MAXC || !(tol > 0.0)) return PPG_ERR_ARG;
    if (r && r->n_total > 0) PPG_TRY(check_roots(r));
    SolveCore c{};
    c.A64 = A;
    c.A32 = nullptr;
    c.roots = r;
    c.b = b;
    c.x = x;
    c.m = m;
    c.tol = tol;
    ppg_default_opts(&c.opts);
    if (opts) c.opts = *opts;
    c.flex = false;
    c.s = (cudaStream_t)stream;
    int32_t rc = run_solve(c);
    if (stats) *stats = c.st;
    return rc;
}

int32_t ppg_solve_flex(const ppg_csr* A64, const ppg_csr* A32, const ppg_roots* r,
                       const double* b, double* x, int32_t m, double tol, const ppg_opts* opts,
                       ppg_stats* stats, void* stream) {
    PPG_TRY(check_csr(A64, PPG_F64));
    PPG_TRY(check_csr(A32, PPG_F32));
    if (A32->n != A64->n || A32->nnz != A64->nnz) return PPG_ERR_ARG;
    if (!b || !x || b == x || m < 1 || m + 1 > ORTHO_MAXC || !(tol > 0.0)) return PPG_ERR_ARG;
    if (r && r->n_total > 0) PPG_TRY(check_roots(r));
    SolveCore c{};
    c.A64 = A64;
    c.A32 = A32;
    c.roots = r;
    c.b = b;
    c.x = x;
    c.m = m;
    c.tol = tol;
    ppg_default_opts(&c.opts);
    if (opts) c.opts = *opts;
    c.flex = true;
    c.s = (cudaStream_t)stream;
    int32_t rc = run_solve(c);
    if (stats) *stats = c.st;
    return rc;
}

int32_t ppg_solve_flex_sweep(const ppg_csr* A64, const ppg_sweep_plan* plan, const ppg_roots* r,
                             const double* b, double* x, int32_t m, double tol,
                             const ppg_opts* opts, ppg_stats* stats, void* stream) {
    PPG_TRY(check_csr(A64, PPG_F64));
    PPG_TRY(check_roots(r));
    if (!plan || sweep_plan_n(plan) != A64->n) return PPG_ERR_ARG;
    if (!b || !x || b == x || m < 1 || m + 1 > ORTHO_MAXC || !(tol > 0.0)) return PPG_ERR_ARG;
    SolveCore c{};
    c.A64 = A64;
    c.A32 = nullptr;
    c.sweep = plan;
    c.roots = r;
    c.b = b;
    c.x = x;
    c.m = m;
    c.tol = tol;
    ppg_default_opts(&c.opts);
    if (opts) c.opts = *opts;
    c.flex = true;
    c.s = (cudaStream_t)stream;
    int32_t rc = run_solve(c);
    if (stats) *stats = c.st;
    return rc;
}

int32_t ppg_solve_double(const ppg_csr* A, const ppg_roots* r1, const ppg_roots* r2,
                         const double* b, double* x, int32_t m, double tol, const ppg_opts* opts,
                         ppg_stats* stats, void* stream) {
    PPG_TRY(check_csr(A, PPG_F64));
    PPG_TRY(check_roots(r1));
    PPG_TRY(check_roots(r2));
    if (!b || !x || b == x || m < 1 || m + 1 > ORTHO_MAXC || !(tol > 0.0)) return PPG_ERR_ARG;
    SolveCore c{};
    c.A64 = A;
    c.roots = r2;
    c.b = b;
    c.x = x;
    c.m = m;
    c.tol = tol;
    ppg_default_opts(&c.opts);
    if (opts) c.opts = *opts;
    if (c.opts.x0_given) return PPG_ERR_ARG;
    c.s = (cudaStream_t)stream;
    const int32_t rc = run_solve_ext(c, r1, 0);
    if (stats) *stats = c.st;
    return rc;
}

int32_t ppg_solve_chpoly(const ppg_csr* A, int32_t d, const double* b, double* x, int32_t m,
                         double tol, const ppg_opts* opts, ppg_stats* stats, void* stream) {
    PPG_TRY(check_csr(A, PPG_F64));
    if (!b || !x || b == x || d < 1 || d + 1 > ORTHO_MAXC || m < 1 || m + 1 > ORTHO_MAXC ||
        !(tol > 0.0))
        return PPG_ERR_ARG;
    SolveCore c{};
    c.A64 = A;
    c.roots = nullptr;
    c.b = b;
    c.x = x;
    c.m = m;
    c.tol = tol;
    ppg_default_opts(&c.opts);
    if (opts) c.opts = *opts;
    if (c.opts.x0_given) return PPG_ERR_ARG;
    c.s = (cudaStream_t)stream;
    const int32_t rc = run_solve_ext(c, nullptr, d);
    if (stats) *stats = c.st;
    return rc;
}

}  // extern "C"

namespace ppg {

// StCh of Section 3.5 with the device vector b: ||r1 - r2||, r1 = b - A p(A) b
// (Algorithm 3 and one SpMV), r2 = pi(A) b (Algorithm 1).  Writes *stch.
static int32_t stch_core(const ppg_csr* A, const ppg_roots* r, const double* b, double* stch,
                         cudaStream_t s) {
    PPG_TRY(setup_device_pool());
    const int32_t n = A->n;
    const int d = r->n_total;
    Arena ar;
    double *y, *r1, *r2, *ba, *bb, *bc, *part, *scal;
    ar.add(&y, n);
    ar.add(&r1, n);
    ar.add(&r2, n);
    ar.add(&ba, n);
    ar.add(&bb, n);
    ar.add(&bc, n);
    ar.add(&part, (size_t)spmv_grid_blocks(n) + 1024);
    ar.add(&scal, 8);
    PPG_TRY(ar.alloc(s));
    struct Guard { Arena& a; cudaStream_t s; ~Guard() { a.release(s); } } guard{ar, s};
    Buffers bufs{};
    bufs.ptr[B_IN] = const_cast<double*>(b);
    bufs.ptr[B_P] = y;
    bufs.ptr[B_A] = ba;
    bufs.ptr[B_B] = bb;
    bufs.ptr[B_C] = bc;
    const double* vals = (const double*)A->vals;
    PPG_TRY(run_plan<double>(plan_p(r->re, r->im, d, false), A->rowptr, A->colind, vals, n,
                             A->nnz, bufs, s, nullptr));
    StepArgs<double> a{};
    a.rowptr = A->rowptr;
    a.colind = A->colind;
    a.vals = vals;
    a.n = n;
    a.flags = keep_a_flag(n, A->nnz, 8, 3);
    a.x = y;
    a.a0 = b;
    a.o0 = r1;
    a.part = part;
    int32_t g = launch_step<double>(OP_RESID, a, s);
    if (g < 0) return g;
    bufs.ptr[B_OUT] = r2;
    PPG_TRY(run_plan<double>(plan_phi(r->re, r->im, d, true), A->rowptr, A->colind, vals, n,
                             A->nnz, bufs, s, nullptr));
    int nparts = 0;
    PPG_TRY(launch_diff_norm2_part(r1, r2, n, part, s, &nparts));
    PPG_TRY(launch_reduce_norm(part, nparts, scal, nullptr, s));
    double sc[8];
    PPG_CUDA(cudaMemcpyAsync(sc, scal, sizeof(sc), cudaMemcpyDeviceToHost, s));
    PPG_CUDA(cudaStreamSynchronize(s));
    *stch = sc[3];
    return std::isfinite(sc[3]) ? PPG_OK : PPG_ERR_NONFINITE;
}

}  // namespace ppg

extern "C" {

int32_t ppg_stability_check(const ppg_csr* A, const ppg_roots* r, const double* b,
                            double* stch, void* stream) {
    PPG_TRY(check_csr(A, PPG_F64));
    PPG_TRY(check_roots(r));
    if (!b || !stch) return PPG_ERR_ARG;
    return stch_core(A, r, b, stch, (cudaStream_t)stream);
}

int32_t ppg_build_poly_checked(const ppg_csr* A, int32_t d, const double* v0, const double* b,
                               double stch_tol, int32_t d_min, const ppg_opts* opts,
                               ppg_roots* out, ppg_poly_check* info, void* stream) {
    PPG_TRY(check_csr(A, PPG_F64));
    if (!v0 || !out || d < 1 || d + 1 > ORTHO_MAXC || !(stch_tol >= 0.0)) return PPG_ERR_ARG;
    ppg_opts o;
    ppg_default_opts(&o);
    if (opts) o = *opts;
    cudaStream_t s = (cudaStream_t)stream;
    const int ldh = d + 1;
    std::vector<double> H((size_t)ldh * d, 0.0);
    // Algorithm 4 step 1 at the requested degree; its Hessenberg matrix also
    // gives every lower degree (GMRES(d') from v0 is its leading block)
    const int32_t built = build_core(A, d, v0, o, nullptr, out, H.data(), s);
    if (built < 0) return built;
    // the check vector u = b / ||b|| (v0 / ||v0|| when b is NULL)
    const int32_t n = A->n;
    Arena ar;
    double *u = nullptr, *part = nullptr, *scal = nullptr;
    ar.add(&u, n);
    ar.add(&part, (size_t)spmv_grid_blocks(n) + 1024);
    ar.add(&scal, 8);
    PPG_TRY(ar.alloc(s));
    struct Guard { Arena& a; cudaStream_t s; ~Guard() { a.release(s); } } guard{ar, s};
    const double* src = b ? b : v0;
    int nparts = 0;
    PPG_TRY(launch_norm2_part(src, n, part, s, &nparts));
    PPG_TRY(launch_reduce_norm(part, nparts, scal, nullptr, s));
    PPG_TRY(launch_scale(src, u, n, scal + 4, s));
    double sc[8];
    PPG_CUDA(cudaMemcpyAsync(sc, scal, sizeof(sc), cudaMemcpyDeviceToHost, s));
    PPG_CUDA(cudaStreamSynchronize(s));
    if (!(sc[3] > 0.0) || !std::isfinite(sc[3])) return PPG_ERR_ARG;
    const int floor_d = std::max(1, std::min<int>(d_min, out->n_orig));
    ppg_poly_check pc{};
    pc.d_requested = d;
    int deg = out->n_orig;
    for (;;) {
        double stch = 0.0;
        const int32_t rc = stch_core(A, out, u, &stch, s);
        if (rc == PPG_ERR_NONFINITE) {
            stch = HUGE_VAL;   // overflowed: as unstable as it gets
        } else if (rc < 0) {
            return rc;
        }
        pc.n_tried += 1;
        if (pc.n_tried == 1) pc.stch_first = stch;
        pc.stch = stch;
        pc.d_chosen = deg;
        if (stch <= stch_tol || deg <= floor_d) break;
        deg = std::max(floor_d, deg / 2);
        const int32_t rr = ppg_roots_from_hessenberg(H.data(), ldh, deg, &o, out);
        if (rr < 0) return rr;
    }
    if (info) *info = pc;
    return built;   // PPG_OK or PPG_LUCKY_BREAKDOWN
}

int32_t ppg_csr_transpose(const ppg_csr* A, int32_t* rowptr_t, int32_t* colind_t, void* vals_t,
                          int32_t* perm, void* stream) {
    PPG_TRY(check_csr(A, -1));
    if (!rowptr_t || (A->nnz > 0 && (!colind_t || !vals_t))) return PPG_ERR_ARG;
    PPG_TRY(setup_device_pool());
    cudaStream_t s = (cudaStream_t)stream;
    Arena ar;
    int32_t* work = nullptr;
    ar.add(&work, 2 * (size_t)A->n + 1);
    PPG_TRY(ar.alloc(s));
    int32_t rc = launch_transpose(A, rowptr_t, colind_t, vals_t, perm, work, s);
    ar.release(s);
    return rc;
}

int32_t ppg_adjoint_vals_grad(const ppg_csr* A, const double* lambda, const double* x,
                              double* gvals, void* stream) {
    PPG_TRY(check_csr(A, PPG_F64));
    if (!lambda || !x || !gvals) return PPG_ERR_ARG;
    return launch_adjoint_grad(A, lambda, x, gvals, (cudaStream_t)stream);
}

}  // extern "C"
