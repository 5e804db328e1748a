// Multi-root fused sweep (matrix-powers style, the communication-avoiding
// idea the paper points to in its introduction): both SpMV passes of one
// conjugate pair of Algorithm 3 in ONE pass over the matrix, in FP32.
//
// A conjugate pair of Algorithm 3 is two SpMV-root steps:
//   P_PAIR1: tmp = 2a prod - A prod ;  p' = p + tmp / (a^2 + b^2)
//   P_PAIR2: prod' = prod - A tmp / (a^2 + b^2)   (or the fused final root)
// The second needs tmp at the neighbours of each row.  After a symmetric
// reordering of A into compact row tiles (a blocked or BFS-grown ordering,
// kept for the life of a plan), one CTA owns a tile of T rows: phase A
// computes tmp over the tile and its halo (the rows outside the tile that
// the tile's rows reference) into shared memory, and p' for the tile's
// rows; phase B computes A tmp for the tile's rows from shared memory.  The
// pair then reads the tile's matrix rows once from HBM (the halo rows'
// entries come with neighbouring tiles' traffic) and never writes tmp.
//
// Every row keeps the unfused kernels' arithmetic exactly: one FP32 FMA per
// nonzero in the row's stored order, the same epilogue forms.  A symmetric
// permutation keeps each row's entries in their order, so the result is
// bit-identical to ppg_apply_poly on the original matrix.
//
// Measured on GB300 (160^3, 16 x 16 x 8 blocks): a pair moves 39 % fewer DRAM
// bytes than the two unfused passes but takes about twice as long -- each
// CTA runs its two phases over a whole tile back to back and the kernel is
// bound by the latency of its gathers -- so the solver's default remains the
// one-pass-per-root chain, and plans are an explicit choice of the caller.
#include <algorithm>
#include <cstring>
#include <vector>

#include "ppg_common.cuh"

struct ppg_sweep_plan {
    int32_t n = 0, nnz = 0, T = 0, ntiles = 0, max_halo = 0, fused = 0;
    int64_t halo_total = 0;
    int dev = 0;
    int32_t* rowptr = nullptr;    // permuted matrix, [n + 1]
    int32_t* colind = nullptr;    // [nnz], columns relabelled, row order kept
    float* vals = nullptr;        // [nnz]
    int32_t* perm = nullptr;      // new row i is original row perm[i]
    int32_t* halo_off = nullptr;  // [ntiles + 1]
    int32_t* halo_idx = nullptr;  // sorted halo rows per tile (new numbering)
    void* mem = nullptr;          // one device allocation holding all of it
};

namespace ppg {
namespace {

constexpr int SW_THREADS = 256;    // threads per CTA; a thread owns two rows of a sub-tile
constexpr int SW_SUB = 2 * SW_THREADS;   // rows per sub-tile
constexpr int SW_CHUNK = 4096;     // nonzeros staged per chunk (32 KB)

// Shared memory of one tile: the staging chunk, tmp over the tile and its
// halo, the halo list.
size_t sweep_smem(int T, int halo) {
    return (size_t)SW_CHUNK * (sizeof(float) + sizeof(int32_t)) +
           (size_t)(T + halo) * sizeof(float) + (size_t)halo * sizeof(int32_t);
}

__device__ __forceinline__ int halo_slot(const int32_t* h, int nh, int32_t c) {
    int lo = 0, hi = nh - 1;
    while (lo < hi) {   // the halo list is sorted and holds c
        const int mid = (lo + hi) >> 1;
        if (h[mid] < c) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void sw_stage(float* sval, int32_t* scol, const float* vals,
                                         const int32_t* colind, int32_t c0, int32_t c1) {
    for (int32_t k = c0 + threadIdx.x; k < c1; k += SW_THREADS) {
        const unsigned sv = (unsigned)__cvta_generic_to_shared(sval + (k - c0));
        const unsigned sc = (unsigned)__cvta_generic_to_shared(scol + (k - c0));
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sv), "l"(vals + k) : "memory");
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sc), "l"(colind + k)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// acc_a / acc_b += the staged products of rows a and b (staged ranges
// [ka, ha) and [kb, hb)), both rows' gathers in flight together, each row
// summed in stored order.  X(c) gives the vector entry of column c.
template <typename XF>
__device__ __forceinline__ void sw_two_rows(const float* sval, const int32_t* scol, int32_t ka,
                                            int32_t ha, int32_t kb, int32_t hb, float& acc_a,
                                            float& acc_b, XF X) {
    for (; ka + 2 <= ha && kb + 2 <= hb; ka += 2, kb += 2) {
        const float xa0 = X(scol[ka]), xa1 = X(scol[ka + 1]);
        const float xb0 = X(scol[kb]), xb1 = X(scol[kb + 1]);
        acc_a = fmaf(sval[ka], xa0, acc_a);
        acc_a = fmaf(sval[ka + 1], xa1, acc_a);
        acc_b = fmaf(sval[kb], xb0, acc_b);
        acc_b = fmaf(sval[kb + 1], xb1, acc_b);
    }
    for (; ka < ha; ++ka) acc_a = fmaf(sval[ka], X(scol[ka]), acc_a);
    for (; kb < hb; ++kb) acc_b = fmaf(sval[kb], X(scol[kb]), acc_b);
}

// One conjugate pair over one tile (see the file comment).  prod = a0 of
// both steps, p = the accumulator (a1 of P_PAIR1, read unless PZERO),
// pout = o0 of P_PAIR1 (p'), qout = o0 of P_PAIR2 (prod', or p'' when
// FINAL: qout = pout then, and p' goes through pout between the phases).
// The tile's rows go in sub-tiles of SW_SUB rows, two per thread, whose
// nonzeros are staged in shared memory by coalesced copies (in chunks, so
// any row length works); each row sums its products in stored order, as
// the unfused kernel does.
__global__ void __launch_bounds__(SW_THREADS)
k_sweep_pair(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
             const float* __restrict__ vals, int32_t n, int T,
             const int32_t* __restrict__ halo_off, const int32_t* __restrict__ halo_idx,
             const float* __restrict__ prod, const float* p, float* pout, float* qout,
             float c1, float c2, float c3, int pzero, int final_) {
    extern __shared__ __align__(16) unsigned char sw_raw[];
    const int tile = blockIdx.x;
    const int32_t lo = tile * T;
    const int rows = min(T, n - lo);
    const int h0 = halo_off[tile], nh = halo_off[tile + 1] - h0;
    float* sval = reinterpret_cast<float*>(sw_raw);
    int32_t* scol = reinterpret_cast<int32_t*>(sval + SW_CHUNK);
    float* tmp_s = reinterpret_cast<float*>(scol + SW_CHUNK);   // [T + nh]
    int32_t* halo_s = reinterpret_cast<int32_t*>(tmp_s + T + nh);
    const int tid = threadIdx.x;
    for (int i = tid; i < nh; i += SW_THREADS) halo_s[i] = halo_idx[h0 + i];
    __syncthreads();   // the halo list is read by other threads below
    auto xprod = [&](int32_t c) { return __ldg(prod + c); };

    // phase A, tile rows: tmp = c1 prod - A prod; p'
    for (int sub = 0; sub < rows; sub += SW_SUB) {
        const int32_t r0 = lo + sub;
        const int nr = min(SW_SUB, rows - sub);
        const int32_t k0 = __ldg(rowptr + r0), k1 = __ldg(rowptr + r0 + nr);
        const int ia = tid, ib = tid + SW_THREADS;
        const int32_t alo = ia < nr ? __ldg(rowptr + r0 + ia) : k1;
        const int32_t ahi = ia < nr ? __ldg(rowptr + r0 + ia + 1) : k1;
        const int32_t blo = ib < nr ? __ldg(rowptr + r0 + ib) : k1;
        const int32_t bhi = ib < nr ? __ldg(rowptr + r0 + ib + 1) : k1;
        float acc_a = 0.f, acc_b = 0.f;
        for (int32_t c0 = k0; c0 < k1; c0 += SW_CHUNK) {
            const int32_t ce = min(k1, c0 + SW_CHUNK);
            sw_stage(sval, scol, vals, colind, c0, ce);
            __syncthreads();
            sw_two_rows(sval, scol, max(alo, c0) - c0, min(ahi, ce) - c0, max(blo, c0) - c0,
                        min(bhi, ce) - c0, acc_a, acc_b, xprod);
            __syncthreads();
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int i = q ? ib : ia;
            if (i < nr) {
                const int32_t g = r0 + i;
                const float tmp = fmaf(c1, __ldg(prod + g), -(q ? acc_b : acc_a));
                tmp_s[sub + i] = tmp;
                pout[g] = pzero ? c2 * tmp : fmaf(c2, tmp, p[g]);
            }
        }
    }
    // phase A, halo rows: the same tmp, two rows per thread from global memory
    for (int li = tid; li < nh; li += 2 * SW_THREADS) {
        const int lj = li + SW_THREADS;
        const int32_t ga = halo_s[li];
        const int32_t gb = lj < nh ? halo_s[lj] : ga;
        int32_t ka = __ldg(rowptr + ga), kb = __ldg(rowptr + gb);
        const int32_t ea = __ldg(rowptr + ga + 1), eb = lj < nh ? __ldg(rowptr + gb + 1) : kb;
        float acc_a = 0.f, acc_b = 0.f;
        for (; ka + 2 <= ea && kb + 2 <= eb; ka += 2, kb += 2) {
            const float xa0 = __ldg(prod + __ldg(colind + ka)), xa1 = __ldg(prod + __ldg(colind + ka + 1));
            const float xb0 = __ldg(prod + __ldg(colind + kb)), xb1 = __ldg(prod + __ldg(colind + kb + 1));
            acc_a = fmaf(__ldg(vals + ka), xa0, acc_a);
            acc_a = fmaf(__ldg(vals + ka + 1), xa1, acc_a);
            acc_b = fmaf(__ldg(vals + kb), xb0, acc_b);
            acc_b = fmaf(__ldg(vals + kb + 1), xb1, acc_b);
        }
        for (; ka < ea; ++ka) acc_a = fmaf(__ldg(vals + ka), __ldg(prod + __ldg(colind + ka)), acc_a);
        for (; kb < eb; ++kb) acc_b = fmaf(__ldg(vals + kb), __ldg(prod + __ldg(colind + kb)), acc_b);
        tmp_s[T + li] = fmaf(c1, __ldg(prod + ga), -acc_a);
        if (lj < nh) tmp_s[T + lj] = fmaf(c1, __ldg(prod + gb), -acc_b);
    }
    __syncthreads();   // tmp complete; p' of the tile written (read back below when FINAL)
    // phase B: prod' = prod - c2 A tmp for the tile's rows, tmp from shared
    // memory (tile columns by offset, halo columns by binary search); the
    // tile's nonzeros are staged again (from L2: this CTA read them just now)
    auto xtmp = [&](int32_t c) {
        return (c >= lo && c < lo + rows) ? tmp_s[c - lo] : tmp_s[T + halo_slot(halo_s, nh, c)];
    };
    for (int sub = 0; sub < rows; sub += SW_SUB) {
        const int32_t r0 = lo + sub;
        const int nr = min(SW_SUB, rows - sub);
        const int32_t k0 = __ldg(rowptr + r0), k1 = __ldg(rowptr + r0 + nr);
        const int ia = tid, ib = tid + SW_THREADS;
        const int32_t alo = ia < nr ? __ldg(rowptr + r0 + ia) : k1;
        const int32_t ahi = ia < nr ? __ldg(rowptr + r0 + ia + 1) : k1;
        const int32_t blo = ib < nr ? __ldg(rowptr + r0 + ib) : k1;
        const int32_t bhi = ib < nr ? __ldg(rowptr + r0 + ib + 1) : k1;
        float acc_a = 0.f, acc_b = 0.f;
        for (int32_t c0 = k0; c0 < k1; c0 += SW_CHUNK) {
            const int32_t ce = min(k1, c0 + SW_CHUNK);
            sw_stage(sval, scol, vals, colind, c0, ce);
            __syncthreads();
            sw_two_rows(sval, scol, max(alo, c0) - c0, min(ahi, ce) - c0, max(blo, c0) - c0,
                        min(bhi, ce) - c0, acc_a, acc_b, xtmp);
            __syncthreads();
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int i = q ? ib : ia;
            if (i < nr) {
                const int32_t g = r0 + i;
                const float prodn = fmaf(-c2, q ? acc_b : acc_a, __ldg(prod + g));
                qout[g] = final_ ? fmaf(c3, prodn, pout[g]) : prodn;
            }
        }
    }
}

// y[i] = x[perm[i]] (cast: FP64 source into the FP32 permuted vector)
template <typename TI>
__global__ void k_gather_perm(const TI* __restrict__ x, const int32_t* __restrict__ perm,
                              float* y, int32_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (float)x[perm[i]];
}

// y[perm[i]] = x[i]
__global__ void k_scatter_perm(const float* __restrict__ x, const int32_t* __restrict__ perm,
                               float* y, int32_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[perm[i]] = x[i];
}

// Greedy BFS region growing: parts of up to T rows, each grown
// breadth-first over the matrix pattern from the lowest-numbered row not
// yet placed.  Returns perm (new -> old).
std::vector<int32_t> bfs_parts(int32_t n, const std::vector<int32_t>& rp,
                               const std::vector<int32_t>& ci, int T) {
    std::vector<int32_t> order;
    order.reserve(n);
    std::vector<char> placed(n, 0), queued(n, 0);
    std::vector<int32_t> q;
    int32_t seed = 0;
    while ((int32_t)order.size() < n) {
        while (placed[seed]) ++seed;
        q.clear();
        q.push_back(seed);
        queued[seed] = 1;
        size_t head = 0;
        int taken = 0;
        while (head < q.size() && taken < T) {
            const int32_t v = q[head++];
            placed[v] = 1;
            order.push_back(v);
            ++taken;
            for (int32_t k = rp[v]; k < rp[v + 1]; ++k) {
                const int32_t u = ci[k];
                if (!placed[u] && !queued[u]) {
                    queued[u] = 1;
                    q.push_back(u);
                }
            }
        }
        for (size_t i = head; i < q.size(); ++i) queued[q[i]] = 0;
        for (size_t i = 0; i < head; ++i) queued[q[i]] = 0;
    }
    return order;
}

int elem_grid_sw(int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, grid_cap(8)));
}

}  // namespace

// The chain of Algorithm 3 on the plan's permuted matrix: every pair
// (P_PAIR1 followed by its P_PAIR2) in one fused launch when the plan
// fuses, every other step by the unfused root-step kernel.
int32_t sweep_run_chain(const ppg_sweep_plan* P, const std::vector<Step>& plan,
                        const Buffers& bufs, cudaStream_t s) {
    const int32_t n = P->n;
    const size_t smem = sweep_smem(P->T, P->max_halo);
    for (size_t i = 0; i < plan.size(); ++i) {
        const Step& st = plan[i];
        if (st.op == -1) {   // degree one: P = c1 v (+ P)
            const bool pz = st.flags & F_PZERO;
            PPG_TRY(launch_axpby<float>((float)st.c1, (const float*)bufs.ptr[st.x],
                                        pz ? 0.f : 1.f, pz ? nullptr : (const float*)bufs.ptr[B_P],
                                        (float*)bufs.ptr[B_P], n, s));
            continue;
        }
        if (P->fused && st.op == OP_P_PAIR1 && i + 1 < plan.size() &&
            plan[i + 1].op == OP_P_PAIR2) {
            const Step& s2 = plan[i + 1];
            const bool fin = s2.flags & F_FINAL;
            k_sweep_pair<<<P->ntiles, SW_THREADS, smem, s>>>(
                P->rowptr, P->colind, P->vals, n, P->T, P->halo_off, P->halo_idx,
                (const float*)bufs.ptr[st.a0],
                (st.flags & F_PZERO) ? nullptr : (const float*)bufs.ptr[st.a1],
                (float*)bufs.ptr[st.o0], fin ? (float*)bufs.ptr[st.o0] : (float*)bufs.ptr[s2.o0],
                (float)st.c1, (float)st.c2, (float)s2.c3, (st.flags & F_PZERO) ? 1 : 0,
                fin ? 1 : 0);
            ++g_launches;
            PPG_TRY(check_launch("k_sweep_pair"));
            ++i;
            continue;
        }
        StepArgs<float> a{};
        a.rowptr = P->rowptr;
        a.colind = P->colind;
        a.vals = P->vals;
        a.n = n;
        a.x = st.x >= 0 ? (const float*)bufs.ptr[st.x] : nullptr;
        a.a0 = st.a0 >= 0 ? (const float*)bufs.ptr[st.a0] : nullptr;
        a.a1 = st.a1 >= 0 ? (const float*)bufs.ptr[st.a1] : nullptr;
        a.a2 = st.a2 >= 0 ? (const float*)bufs.ptr[st.a2] : nullptr;
        a.o0 = st.o0 >= 0 ? (float*)bufs.ptr[st.o0] : nullptr;
        a.o1 = st.o1 >= 0 ? (float*)bufs.ptr[st.o1] : nullptr;
        a.c1 = (float)st.c1;
        a.c2 = (float)st.c2;
        a.c3 = (float)st.c3;
        a.flags = st.flags;
        const int32_t g = launch_step<float>(st.op, a, s);
        if (g < 0) return g;
    }
    return PPG_OK;
}

int32_t sweep_gather(const ppg_sweep_plan* P, const void* x, bool x_f64, float* y,
                     cudaStream_t s) {
    if (x_f64)
        k_gather_perm<double><<<elem_grid_sw(P->n), 256, 0, s>>>((const double*)x, P->perm, y,
                                                                 P->n);
    else
        k_gather_perm<float><<<elem_grid_sw(P->n), 256, 0, s>>>((const float*)x, P->perm, y,
                                                                P->n);
    ++g_launches;
    return check_launch("k_gather_perm");
}

int32_t sweep_scatter(const ppg_sweep_plan* P, const float* x, float* y, cudaStream_t s) {
    k_scatter_perm<<<elem_grid_sw(P->n), 256, 0, s>>>(x, P->perm, y, P->n);
    ++g_launches;
    return check_launch("k_scatter_perm");
}

int32_t sweep_plan_n(const ppg_sweep_plan* P) { return P ? P->n : -1; }

// Unique bytes of the chain: every unfused step as step_bytes counts it;
// a fused pair reads the CSR once and touches prod, p (unless it starts
// at zero) and its two outputs once (tmp never reaches memory).
double sweep_chain_bytes(const ppg_sweep_plan* P, const std::vector<Step>& plan) {
    const double M = (double)P->nnz * 8.0 + 4.0 * (double)(P->n + 1);
    double by = 0.0;
    for (size_t i = 0; i < plan.size(); ++i) {
        const Step& st = plan[i];
        if (st.op == -1) {
            by += 4.0 * P->n * ((st.flags & F_PZERO) ? 2 : 3);
            continue;
        }
        if (P->fused && st.op == OP_P_PAIR1 && i + 1 < plan.size() &&
            plan[i + 1].op == OP_P_PAIR2) {
            const bool fin = plan[i + 1].flags & F_FINAL;
            const int vec = 1 + ((st.flags & F_PZERO) ? 0 : 1) + (fin ? 1 : 2);
            by += M + 4.0 * P->n * vec;
            ++i;
            continue;
        }
        by += step_bytes(st.op, st.flags, P->n, P->nnz, 4);
    }
    return by;
}

int64_t sweep_chain_launches(const ppg_sweep_plan* P, const std::vector<Step>& plan) {
    int64_t L = 0;
    for (size_t i = 0; i < plan.size(); ++i, ++L)
        if (P->fused && plan[i].op == OP_P_PAIR1 && i + 1 < plan.size() &&
            plan[i + 1].op == OP_P_PAIR2)
            ++i;
    return L;
}

}  // namespace ppg

using namespace ppg;

extern "C" {

int32_t ppg_sweep_plan_create(const ppg_csr* A, const int32_t* perm_host, int32_t tile_rows,
                              int32_t fuse, ppg_sweep_plan** out, void* stream) {
    if (!out) return PPG_ERR_ARG;
    *out = nullptr;
    PPG_TRY(check_csr(A, PPG_F32));
    if (tile_rows < 32 || tile_rows > 16384 || (tile_rows % 32) != 0) return PPG_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t n = A->n, nnz = A->nnz;
    const int T = tile_rows;
    std::vector<int32_t> rp(n + 1), ci(nnz);
    std::vector<float> va(nnz);
    PPG_CUDA(cudaMemcpyAsync(rp.data(), A->rowptr, sizeof(int32_t) * (n + 1),
                             cudaMemcpyDeviceToHost, s));
    if (nnz > 0) {
        PPG_CUDA(cudaMemcpyAsync(ci.data(), A->colind, sizeof(int32_t) * nnz,
                                 cudaMemcpyDeviceToHost, s));
        PPG_CUDA(cudaMemcpyAsync(va.data(), A->vals, sizeof(float) * nnz,
                                 cudaMemcpyDeviceToHost, s));
    }
    PPG_CUDA(cudaStreamSynchronize(s));
    if (ppg_csr_validate_host(n, nnz, rp.data(), ci.data()) != PPG_OK) return PPG_ERR_CSR;
    // the ordering: the caller's, or BFS-grown parts of T rows
    std::vector<int32_t> perm;
    if (perm_host) {
        perm.assign(perm_host, perm_host + n);
        std::vector<char> seen(n, 0);
        for (int32_t i = 0; i < n; ++i) {
            if (perm[i] < 0 || perm[i] >= n || seen[perm[i]]) return PPG_ERR_ARG;
            seen[perm[i]] = 1;
        }
    } else {
        perm = bfs_parts(n, rp, ci, T);
    }
    std::vector<int32_t> iperm(n);
    for (int32_t i = 0; i < n; ++i) iperm[perm[i]] = i;
    // the permuted matrix: row i is original row perm[i] with its entries in
    // their stored order, columns relabelled
    std::vector<int32_t> prp(n + 1), pci(nnz);
    std::vector<float> pva(nnz);
    prp[0] = 0;
    for (int32_t i = 0; i < n; ++i) {
        const int32_t o = perm[i];
        int32_t k = prp[i];
        for (int32_t e = rp[o]; e < rp[o + 1]; ++e, ++k) {
            pci[k] = iperm[ci[e]];
            pva[k] = va[e];
        }
        prp[i + 1] = k;
    }
    // halo of each tile: the rows outside it that its rows reference
    const int32_t ntiles = (n + T - 1) / T;
    std::vector<int32_t> hoff(ntiles + 1, 0), hidx;
    std::vector<int32_t> buf;
    int max_halo = 0;
    for (int32_t t = 0; t < ntiles; ++t) {
        const int32_t lo = t * T, hi = std::min(n, lo + T);
        buf.clear();
        for (int32_t k = prp[lo]; k < prp[hi]; ++k)
            if (pci[k] < lo || pci[k] >= hi) buf.push_back(pci[k]);
        std::sort(buf.begin(), buf.end());
        buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
        hidx.insert(hidx.end(), buf.begin(), buf.end());
        hoff[t + 1] = (int32_t)hidx.size();
        max_halo = std::max<int>(max_halo, (int)buf.size());
    }
    ppg_sweep_plan* P = new ppg_sweep_plan();
    P->n = n;
    P->nnz = nnz;
    P->T = T;
    P->ntiles = ntiles;
    P->max_halo = max_halo;
    P->halo_total = (int64_t)hidx.size();
    PPG_CUDA(cudaGetDevice(&P->dev));
    // fuse when the halo is at most 60 % of the rows (beyond that the
    // redundant phase-A rows eat the saving) and the tile fits in shared
    // memory
    int smem_max = 0;
    PPG_CUDA(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->dev));
    const size_t need = sweep_smem(T, max_halo);
    P->fused = (fuse != 0 && (double)P->halo_total <= 0.6 * (double)n &&
                need <= (size_t)smem_max) ? 1 : 0;
    // one device allocation, owned by the plan
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t b_rp = al(sizeof(int32_t) * (n + 1)), b_ci = al(sizeof(int32_t) * std::max(nnz, 1));
    const size_t b_va = al(sizeof(float) * std::max(nnz, 1)), b_pm = al(sizeof(int32_t) * n);
    const size_t b_ho = al(sizeof(int32_t) * (ntiles + 1));
    const size_t b_hi = al(sizeof(int32_t) * std::max<size_t>(hidx.size(), 1));
    const cudaError_t e = cudaMalloc(&P->mem, b_rp + b_ci + b_va + b_pm + b_ho + b_hi);
    if (e != cudaSuccess) {
        set_cuda_error(e, "cudaMalloc(sweep plan)");
        cudaGetLastError();
        delete P;
        return PPG_ERR_NOMEM;
    }
    char* m = (char*)P->mem;
    P->rowptr = (int32_t*)m; m += b_rp;
    P->colind = (int32_t*)m; m += b_ci;
    P->vals = (float*)m; m += b_va;
    P->perm = (int32_t*)m; m += b_pm;
    P->halo_off = (int32_t*)m; m += b_ho;
    P->halo_idx = (int32_t*)m;
    int32_t rc = PPG_OK;
    auto up = [&](void* d, const void* h, size_t b) {
        if (rc == PPG_OK && b > 0) {
            const cudaError_t ee = cudaMemcpyAsync(d, h, b, cudaMemcpyHostToDevice, s);
            if (ee != cudaSuccess) { set_cuda_error(ee, "cudaMemcpyAsync(sweep plan)"); rc = PPG_ERR_CUDA; }
        }
    };
    up(P->rowptr, prp.data(), sizeof(int32_t) * (n + 1));
    up(P->colind, pci.data(), sizeof(int32_t) * nnz);
    up(P->vals, pva.data(), sizeof(float) * nnz);
    up(P->perm, perm.data(), sizeof(int32_t) * n);
    up(P->halo_off, hoff.data(), sizeof(int32_t) * (ntiles + 1));
    up(P->halo_idx, hidx.data(), sizeof(int32_t) * hidx.size());
    if (rc == PPG_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = PPG_ERR_CUDA;
    if (rc == PPG_OK && P->fused &&
        cudaFuncSetAttribute(k_sweep_pair, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)need) != cudaSuccess) {
        cudaGetLastError();
        P->fused = 0;
    }
    if (rc != PPG_OK) {
        cudaFree(P->mem);
        delete P;
        return rc;
    }
    *out = P;
    return PPG_OK;
}

int32_t ppg_sweep_plan_info(const ppg_sweep_plan* P, ppg_sweep_info* info) {
    if (!P || !info) return PPG_ERR_ARG;
    info->n = P->n;
    info->nnz = P->nnz;
    info->tile_rows = P->T;
    info->ntiles = P->ntiles;
    info->max_halo = P->max_halo;
    info->fused = P->fused;
    info->halo_total = P->halo_total;
    info->halo_fraction = P->n > 0 ? (double)P->halo_total / (double)P->n : 0.0;
    return PPG_OK;
}

void ppg_sweep_plan_destroy(ppg_sweep_plan* P) {
    if (!P) return;
    if (P->mem) cudaFree(P->mem);
    delete P;
}

int32_t ppg_apply_poly_sweep(const ppg_sweep_plan* P, const ppg_roots* r, const void* v,
                             void* y, void* stream) {
    if (!P || !v || !y || v == y) return PPG_ERR_ARG;
    PPG_TRY(check_roots(r));
    PPG_TRY(setup_device_pool());
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t n = P->n;
    Arena ar;
    float *vh = nullptr, *yh = nullptr, *ba = nullptr, *bb = nullptr, *bc = nullptr;
    ar.add(&vh, n);
    ar.add(&yh, n);
    ar.add(&ba, n);
    ar.add(&bb, n);
    ar.add(&bc, n);
    PPG_TRY(ar.alloc(s));
    struct Guard { Arena& a; cudaStream_t s; ~Guard() { a.release(s); } } guard{ar, s};
    PPG_TRY(sweep_gather(P, v, false, vh, s));
    Buffers bufs{};
    bufs.ptr[B_IN] = vh;
    bufs.ptr[B_OUT] = yh;
    bufs.ptr[B_P] = yh;
    bufs.ptr[B_A] = ba;
    bufs.ptr[B_B] = bb;
    bufs.ptr[B_C] = bc;
    PPG_TRY(sweep_run_chain(P, plan_p(r->re, r->im, r->n_total, false), bufs, s));
    return sweep_scatter(P, yh, (float*)y, s);
}

}  // extern "C"
