// Host FP64 steps of the polynomial construction (Algorithm 4 step 1(b)-(c)
// and Algorithm 2): harmonic Ritz values from the Arnoldi Hessenberg matrix,
// modified Leja ordering, pof and root adding.  These act on d x d data
// (d = polynomial degree) once per polynomial, so they run on the CPU.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <limits>
#include <vector>

#include "ppg_common.cuh"

namespace ppg {

namespace {

// ---------------------------------------------------------------------------
// Eigenvalues of a real upper Hessenberg matrix: implicit double-shift
// (Francis) QR iteration with Householder reflectors of order 3, deflation
// on negligible subdiagonal entries, and an ad hoc shift every tenth
// iteration on a block that does not converge (Golub & Van Loan, Matrix
// Computations, Section 7.5).  Only eigenvalues are needed, so reflectors
// are applied to the active diagonal block alone.
// ---------------------------------------------------------------------------

struct Mat {
    int n;
    std::vector<double> a;  // row-major
    double& operator()(int i, int j) { return a[(size_t)i * n + j]; }
};

// Reflector P = I - beta v v^T with P u = alpha e1, for u of length 2 or 3.
static bool householder(int len, const double* u, double* v, double* beta) {
    double s = 0.0;
    for (int i = 0; i < len; ++i) s += u[i] * u[i];
    double nrm = std::sqrt(s);
    if (nrm == 0.0) return false;
    double alpha = (u[0] >= 0.0) ? -nrm : nrm;
    v[0] = u[0] - alpha;
    for (int i = 1; i < len; ++i) v[i] = u[i];
    double vv = v[0] * v[0];
    for (int i = 1; i < len; ++i) vv += v[i] * v[i];
    if (vv == 0.0) return false;
    *beta = 2.0 / vv;
    return true;
}

// eigenvalues of [[a, b], [c, d]]
static void eig2x2(double a, double b, double c, double d, double* wr1, double* wi1,
                   double* wr2, double* wi2) {
    double p = 0.5 * (a - d);
    double bc = b * c;
    double disc = p * p + bc;
    if (disc >= 0.0) {
        double sq = std::sqrt(disc);
        double z = p + (p >= 0.0 ? sq : -sq);
        *wr1 = d + z;
        *wr2 = (z != 0.0) ? d - bc / z : d + z;
        *wi1 = 0.0;
        *wi2 = 0.0;
    } else {
        double sq = std::sqrt(-disc);
        *wr1 = d + p;
        *wr2 = d + p;
        *wi1 = sq;
        *wi2 = -sq;
    }
}

static int32_t hessenberg_eig(Mat& H, double* wr, double* wi) {
    const int n = H.n;
    const double eps = DBL_EPSILON;
    double anorm = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = std::max(i - 1, 0); j < n; ++j) anorm += std::fabs(H(i, j));
    if (!std::isfinite(anorm)) return PPG_ERR_NONFINITE;
    int hi = n - 1;
    int its = 0;
    while (hi >= 0) {
        int l = hi;
        while (l > 0) {
            double s = std::fabs(H(l - 1, l - 1)) + std::fabs(H(l, l));
            if (s == 0.0) s = anorm;
            if (std::fabs(H(l, l - 1)) <= eps * s) {
                H(l, l - 1) = 0.0;
                break;
            }
            --l;
        }
        if (l == hi) {
            wr[hi] = H(hi, hi);
            wi[hi] = 0.0;
            --hi;
            its = 0;
            continue;
        }
        if (l == hi - 1) {
            eig2x2(H(hi - 1, hi - 1), H(hi - 1, hi), H(hi, hi - 1), H(hi, hi),
                   &wr[hi - 1], &wi[hi - 1], &wr[hi], &wi[hi]);
            hi -= 2;
            its = 0;
            continue;
        }
        if (its >= 60) return PPG_ERR_EIG;
        ++its;
        // shift polynomial z^2 - s z + t
        double s, t;
        if (its % 10 == 0) {
            double x = std::fabs(H(hi, hi - 1)) + std::fabs(H(hi - 1, hi - 2));
            s = 1.5 * x;
            t = x * x;
        } else {
            s = H(hi - 1, hi - 1) + H(hi, hi);
            t = H(hi - 1, hi - 1) * H(hi, hi) - H(hi - 1, hi) * H(hi, hi - 1);
        }
        // first column of H^2 - s H + t I on rows l..l+2
        double u[3];
        u[0] = H(l, l) * H(l, l) + H(l, l + 1) * H(l + 1, l) - s * H(l, l) + t;
        u[1] = H(l + 1, l) * (H(l, l) + H(l + 1, l + 1) - s);
        u[2] = H(l + 1, l) * H(l + 2, l + 1);
        for (int k = l; k <= hi - 2; ++k) {
            double v[3], beta;
            if (householder(3, u, v, &beta)) {
                int c0 = std::max(l, k - 1);
                for (int j = c0; j <= hi; ++j) {
                    double dot = beta * (v[0] * H(k, j) + v[1] * H(k + 1, j) + v[2] * H(k + 2, j));
                    H(k, j) -= dot * v[0];
                    H(k + 1, j) -= dot * v[1];
                    H(k + 2, j) -= dot * v[2];
                }
                int r1 = std::min(k + 3, hi);
                for (int i = l; i <= r1; ++i) {
                    double dot = beta * (H(i, k) * v[0] + H(i, k + 1) * v[1] + H(i, k + 2) * v[2]);
                    H(i, k) -= dot * v[0];
                    H(i, k + 1) -= dot * v[1];
                    H(i, k + 2) -= dot * v[2];
                }
                if (k > l) {
                    H(k + 1, k - 1) = 0.0;
                    H(k + 2, k - 1) = 0.0;
                }
            }
            u[0] = H(k + 1, k);
            u[1] = H(k + 2, k);
            if (k < hi - 2) u[2] = H(k + 3, k);
        }
        double v[2], beta;
        if (householder(2, u, v, &beta)) {
            int k = hi - 1;
            for (int j = std::max(l, k - 1); j <= hi; ++j) {
                double dot = beta * (v[0] * H(k, j) + v[1] * H(k + 1, j));
                H(k, j) -= dot * v[0];
                H(k + 1, j) -= dot * v[1];
            }
            for (int i = l; i <= hi; ++i) {
                double dot = beta * (H(i, k) * v[0] + H(i, k + 1) * v[1]);
                H(i, k) -= dot * v[0];
                H(i, k + 1) -= dot * v[1];
            }
            if (k - 1 > l) H(k + 1, k - 1) = 0.0;
        }
    }
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(wr[i]) || !std::isfinite(wi[i])) return PPG_ERR_NONFINITE;
    return PPG_OK;
}

// solve M x = rhs (n x n, row-major, destroyed) by Gaussian elimination
// with partial pivoting
static int32_t lu_solve(int n, std::vector<double>& M, std::vector<double>& rhs) {
    for (int k = 0; k < n; ++k) {
        int piv = k;
        double best = std::fabs(M[(size_t)k * n + k]);
        for (int i = k + 1; i < n; ++i) {
            double v = std::fabs(M[(size_t)i * n + k]);
            if (v > best) { best = v; piv = i; }
        }
        if (best == 0.0) return PPG_ERR_SINGULAR_H;
        if (piv != k) {
            for (int j = 0; j < n; ++j) std::swap(M[(size_t)k * n + j], M[(size_t)piv * n + j]);
            std::swap(rhs[k], rhs[piv]);
        }
        double dkk = M[(size_t)k * n + k];
        for (int i = k + 1; i < n; ++i) {
            double f = M[(size_t)i * n + k] / dkk;
            if (f == 0.0) continue;
            for (int j = k; j < n; ++j) M[(size_t)i * n + j] -= f * M[(size_t)k * n + j];
            rhs[i] -= f * rhs[k];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = rhs[i];
        for (int j = i + 1; j < n; ++j) s -= M[(size_t)i * n + j] * rhs[j];
        rhs[i] = s / M[(size_t)i * n + i];
    }
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(rhs[i])) return PPG_ERR_SINGULAR_H;
    return PPG_OK;
}

struct Unit {
    double re, im;   // representative (+Im member for a pair)
};

static double dist(double ar, double ai, double br, double bi) {
    return std::hypot(ar - br, ai - bi);
}

}  // namespace

// theta = eig(H_dd + h_{d+1,d}^2 f e_d^T), H_dd^T f = e_d
int32_t host_harmonic_ritz(const double* Hbar, int ldh, int d, double* re, double* im) {
    if (!Hbar || !re || !im || d < 1 || ldh < d) return PPG_ERR_ARG;
    // H_dd^T f = e_d: (H^T)(i, j) = H(j, i) = Hbar[i*ldh + j]
    std::vector<double> M((size_t)d * d), f(d, 0.0);
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) M[(size_t)i * d + j] = Hbar[(size_t)i * ldh + j];
    for (int i = 0; i < d * d; ++i)
        if (!std::isfinite(M[i])) return PPG_ERR_NONFINITE;
    f[d - 1] = 1.0;
    double h = (ldh > d) ? Hbar[(size_t)(d - 1) * ldh + d] : 0.0;
    int32_t rc = lu_solve(d, M, f);
    if (rc != PPG_OK) return rc;
    Mat G;
    G.n = d;
    G.a.assign((size_t)d * d, 0.0);
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) G(i, j) = Hbar[(size_t)j * ldh + i];
    for (int i = 0; i < d; ++i) G(i, d - 1) += h * h * f[i];
    // G stays upper Hessenberg: the update only touches the last column
    return hessenberg_eig(G, re, im);
}

// Modified Leja ordering
int32_t host_leja(int k, const double* re, const double* im, double* ro, double* io) {
    if (k < 0 || (k > 0 && (!re || !im || !ro || !io))) return PPG_ERR_ARG;
    int npos = 0, nneg = 0;
    std::vector<Unit> rem;
    for (int i = 0; i < k; ++i) {
        if (!std::isfinite(re[i]) || !std::isfinite(im[i])) return PPG_ERR_NONFINITE;
        if (im[i] > 0) ++npos;
        if (im[i] < 0) ++nneg;
        if (im[i] >= 0) rem.push_back({re[i], im[i]});
    }
    if (npos != nneg) return PPG_ERR_ARG;
    std::vector<Unit> chosen;   // both members of pairs
    int out = 0;
    const double NEG_INF = -std::numeric_limits<double>::infinity();
    while (!rem.empty()) {
        int best = -1;
        double bs = 0, br = 0, bi = 0;
        for (size_t c = 0; c < rem.size(); ++c) {
            const Unit& z = rem[c];
            double score;
            if (chosen.empty()) {
                double m = std::hypot(z.re, z.im);
                score = (m > 0) ? std::log(m) : NEG_INF;
            } else {
                score = 0.0;
                for (const Unit& q : chosen) {
                    double dd = dist(z.re, z.im, q.re, q.im);
                    score += (dd > 0) ? std::log(dd) : NEG_INF;
                }
            }
            bool better;
            if (best < 0) better = true;
            else if (score != bs) better = score > bs;
            else if (z.re != br) better = z.re > br;
            else better = z.im > bi;
            if (better) { best = (int)c; bs = score; br = z.re; bi = z.im; }
        }
        Unit u = rem[best];
        rem.erase(rem.begin() + best);
        chosen.push_back(u);
        ro[out] = u.re; io[out] = u.im; ++out;
        if (u.im != 0) {
            chosen.push_back({u.re, -u.im});
            ro[out] = u.re; io[out] = -u.im; ++out;
        }
    }
    return PPG_OK;
}

// Algorithm 2 steps 2-3
int32_t host_add_roots(int k, const double* re, const double* im, double thr,
                       double step, ppg_roots* out) {
    if (!out || k < 1 || !re || !im) return PPG_ERR_ARG;
    // log10 pof over the k original roots: |1 - t_k/t_i| = |t_i - t_k| / |t_i|
    std::vector<double> lpof(k);
    for (int a = 0; a < k; ++a) {
        double s = 0.0;
        for (int i = 0; i < k; ++i) {
            if (i == a) continue;
            double m = dist(re[i], im[i], re[a], im[a]) / std::hypot(re[i], im[i]);
            s += (m > 0) ? std::log10(m) : -std::numeric_limits<double>::infinity();
        }
        lpof[a] = s;
    }
    // units with their pof
    struct U { double re, im, lp; int id; };
    std::vector<U> units;
    for (int a = 0; a < k;) {
        if (im[a] != 0) {
            if (a + 1 >= k || re[a + 1] != re[a] || im[a + 1] != -im[a]) return PPG_ERR_ARG;
            units.push_back({re[a], im[a], lpof[a], (int)units.size()});
            a += 2;
        } else {
            units.push_back({re[a], 0.0, lpof[a], (int)units.size()});
            a += 1;
        }
    }
    std::vector<U> lst = units;   // copies get id -1
    int n_added = 0;
    for (size_t uid = 0; uid < units.size(); ++uid) {
        double x = (units[uid].lp - thr) / step;
        int c = (x > 0) ? (int)std::ceil(x) : 0;
        if (c == 0) continue;
        U cp = units[uid];
        cp.id = -1;
        lst.push_back(cp);
        int p = 0;
        while (lst[p].id != (int)uid) ++p;
        int L = (int)lst.size();
        int span = (L - 1) - p;
        for (int j = c - 1; j >= 1; --j) {
            int off = (int)std::floor((double)(j * span) / c + 0.5);
            int q = p + std::max(1, off);
            lst.insert(lst.begin() + q, cp);
        }
        n_added += c * (units[uid].im != 0 ? 2 : 1);
    }
    int total = 0;
    for (const U& u : lst) total += (u.im != 0) ? 2 : 1;
    out->n_orig = k;
    out->n_added = n_added;
    out->n_total = total;
    if (out->log10_pof) {
        if (out->capacity < k) return PPG_ERR_CAPACITY;
        for (int a = 0; a < k; ++a) out->log10_pof[a] = lpof[a];
    }
    if (total > out->capacity || !out->re || !out->im) return PPG_ERR_CAPACITY;
    int o = 0;
    for (const U& u : lst) {
        out->re[o] = u.re; out->im[o] = u.im; ++o;
        if (u.im != 0) { out->re[o] = u.re; out->im[o] = -u.im; ++o; }
    }
    return PPG_OK;
}

}  // namespace ppg
