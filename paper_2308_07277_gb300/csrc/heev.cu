// Lowest eigenpairs of a complex Hermitian matrix in FP64, for the Rayleigh-Ritz step of the
// Davidson solver (and the Loewdin orthonormalisation).  Classical dense algorithms, written
// for a GPU whose FP64 rate is low: the O(m^3) work is done once (Householder reduction), and
// only the wanted eigenpairs are computed from the tridiagonal matrix.
//
//   1. k_tridiag_rows Householder reduction Q^H A Q = T, T real symmetric tridiagonal
//                     (Golub & Van Loan, Matrix Computations, Sec. 8.3.1; the complex
//                     reflector makes every subdiagonal element real).  One cooperative
//                     launch, one grid barrier per column, rows resident in shared memory
//                     (k_tridiag: two barriers per column, for matrices beyond that).
//   2. k_multisect    the j-th smallest eigenvalue of T by multisection on Sturm counts
//                     (Sec. 8.4.1): a warp tests 32 points per round, 12 rounds.
//   3. k_inviter      eigenvectors of T by inverse iteration (LU with partial pivoting of the
//                     tridiagonal, three solves), one warp per eigenvalue; k_cluster_orth
//                     then orthonormalises the vectors of each cluster of close eigenvalues
//                     by Gram-Schmidt (Sec. 8.4.2, 8.2.2).
//   4. k_backtransf   y <- Q y by applying the reflectors in reverse order, one CTA per
//                     eigenvector (no grid barrier needed: the columns are independent).
#include <cooperative_groups.h>

#include <algorithm>

#include <map>
#include <mutex>

#include "qm_internal.h"

namespace cg = cooperative_groups;

namespace qm {
namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // conj(a) * b
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// block-wide sum of a double2 (every thread gets the result); sh >= 32 entries
__device__ double2 block_sum2(double2 v, double2* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double2 t = make_double2(0.0, 0.0);
    for (int i = 0; i < nw; ++i) {  // fixed order: identical result in every block
        t.x += sh[i].x;
        t.y += sh[i].y;
    }
    return t;
}

__global__ void __launch_bounds__(256)
k_tridiag(double2* __restrict__ A, int lda, int m, double2* __restrict__ Vh, double2* __restrict__ tau,
          double* __restrict__ d, double* __restrict__ e, double2* __restrict__ wbuf) {
    cg::grid_group grid = cg::this_grid();
    extern __shared__ double2 sm[];
    double2* sv = sm;       // reflector v (length n)
    double2* sw = sm + m;   // w
    __shared__ double2 red[32];
    const int tid = threadIdx.x, bs = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int gw = blockIdx.x * (bs >> 5) + warp, nwg = gridDim.x * (bs >> 5);
    for (int k = 0; k < m - 1; ++k) {
        const int n = m - k - 1;
        for (int i = tid; i < n; i += bs) sv[i] = A[(size_t)(k + 1 + i) * lda + k];
        __syncthreads();
        double part = 0.0;
        for (int i = 1 + tid; i < n; i += bs) part += sv[i].x * sv[i].x + sv[i].y * sv[i].y;
        const double xn2 = block_sum2(make_double2(part, 0.0), red).x;
        const double2 alpha = sv[0];
        double2 t = make_double2(0.0, 0.0), scale = make_double2(0.0, 0.0);
        double beta = alpha.x;
        if (xn2 > 0.0 || alpha.y != 0.0) {
            // complex reflector H = I - t v v^H with H^H (alpha, x) = (beta, 0), beta real
            beta = -copysign(sqrt(alpha.x * alpha.x + alpha.y * alpha.y + xn2), alpha.x);
            t = make_double2((beta - alpha.x) / beta, -alpha.y / beta);
            const double2 den = make_double2(alpha.x - beta, alpha.y);  // 1 / (alpha - beta)
            const double dd = den.x * den.x + den.y * den.y;
            scale = make_double2(den.x / dd, -den.y / dd);
        }
        __syncthreads();
        for (int i = tid; i < n; i += bs) sv[i] = (i == 0) ? make_double2(1.0, 0.0) : cmul(sv[i], scale);
        __syncthreads();
        if (blockIdx.x == 0) {
            for (int i = tid; i < n; i += bs) Vh[(size_t)k * m + k + 1 + i] = sv[i];
            if (tid == 0) {
                tau[k] = t;
                e[k] = beta;
                d[k] = A[(size_t)k * lda + k].x;
            }
        }
        if (t.x == 0.0 && t.y == 0.0) continue;  // uniform: every block computed the same t
        // w = t * A22 v, one warp per row
        for (int r = gw; r < n; r += nwg) {
            const double2* row = A + (size_t)(k + 1 + r) * lda + (k + 1);
            double2 acc = make_double2(0.0, 0.0);
            for (int j = lane; j < n; j += 32) {
                const double2 a = row[j], v = sv[j];
                acc.x += a.x * v.x - a.y * v.y;
                acc.y += a.x * v.y + a.y * v.x;
            }
            for (int o = 16; o > 0; o >>= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
            }
            if (lane == 0) wbuf[r] = cmul(t, acc);
        }
        grid.sync();
        for (int i = tid; i < n; i += bs) sw[i] = wbuf[i];
        __syncthreads();
        double2 dp = make_double2(0.0, 0.0);
        for (int i = tid; i < n; i += bs) {
            const double2 c = cmulc(sw[i], sv[i]);  // w^H v
            dp.x += c.x;
            dp.y += c.y;
        }
        dp = block_sum2(dp, red);
        const double2 a2 = cmul(make_double2(-0.5 * t.x, -0.5 * t.y), dp);
        for (int i = tid; i < n; i += bs) {
            const double2 av = cmul(a2, sv[i]);
            sw[i].x += av.x;
            sw[i].y += av.y;
        }
        __syncthreads();
        // A22 -= v w^H + w v^H, one row per block iteration
        for (int i = blockIdx.x; i < n; i += gridDim.x) {
            double2* row = A + (size_t)(k + 1 + i) * lda + (k + 1);
            const double2 vi = sv[i], wi = sw[i];
            for (int j = tid; j < n; j += bs) {
                const double2 vj = sv[j], wj = sw[j];
                double2 a = row[j];
                // v_i conj(w_j) + w_i conj(v_j)
                a.x -= vi.x * wj.x + vi.y * wj.y + wi.x * vj.x + wi.y * vj.y;
                a.y -= vi.y * wj.x - vi.x * wj.y + wi.y * vj.x - wi.x * vj.y;
                row[j] = a;
            }
        }
        grid.sync();
    }
    if (blockIdx.x == 0 && tid == 0) d[m - 1] = A[(size_t)(m - 1) * lda + (m - 1)].x;
}

// The same reduction with one grid barrier per column.  Row i of A is owned by CTA i mod G
// and, when the rows fit (kSmemRows), lives in that CTA's shared memory for the whole
// reduction.  Step k needs row k of A^(k) (A after the first k reflections): its owner
// publishes row k of A^(k-1) one step early, and every CTA applies the rank-2 update of step
// k-1 to that copy itself, so the pivot row costs no extra barrier.  Per step, every CTA:
//   1. forms the pivot row and the reflector (v_k, t_k) redundantly (same data, same order:
//      bitwise identical in every CTA);
//   2. applies the update of step k-1 to its own rows (columns > k) and multiplies them by
//      v_k, writing its entries of w_k = t_k A22 v_k; the owner of row k+1 publishes it;
//   3. grid barrier;
//   4. reads w_k and applies the symmetric correction w_k -= (t_k/2)(w_k^H v_k) v_k.
// w and the published row are double-buffered by step parity: a CTA may already write step
// k+1's entries while another still reads step k's (the barrier of step k+1 orders step k+2).
// The arithmetic per element is that of k_tridiag (same reflector, same update formula).
template <bool kSmemRows>
__global__ void __launch_bounds__(256)
k_tridiag_rows(double2* __restrict__ A, int lda, int m, double2* __restrict__ Vh, double2* __restrict__ tau,
               double* __restrict__ d, double* __restrict__ e, double2* __restrict__ wbuf, double2* __restrict__ prow) {
    cg::grid_group grid = cg::this_grid();
    extern __shared__ double2 sm[];
    double2* sv = sm;             // v_k (indices k+1..m-1)
    double2* svp = sm + m;        // v_{k-1}
    double2* sw = sm + 2 * m;     // w_{k-1}
    double2* sr = sm + 3 * m;     // pivot row of step k
    double2* srows = sm + 4 * m;  // own rows (kSmemRows)
    __shared__ double2 red[32];
    __shared__ double2 s_sc[3];          // t, scale, beta of the current reflector
    __shared__ double2 s_part[8][8];     // per-warp partial products of up to 8 own rows
    const int tid = threadIdx.x, bs = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int G = gridDim.x, b = blockIdx.x;
    const int nr = b < m ? (m - b + G - 1) / G : 0;  // own rows i = b + G r, r < nr
    if (kSmemRows)
        for (int r = 0; r < nr; ++r)
            for (int j = tid; j < m; j += bs) srows[(size_t)r * m + j] = A[(size_t)(b + G * r) * lda + j];
    __syncthreads();
    bool have_prev = false;  // svp, sw hold the update of the previous step
    for (int k = 0; k < m - 1; ++k) {
        // 1. pivot row r_j = A^(k)[k][j], j >= k
        const double2* P = k == 0 ? A : prow + (size_t)(k & 1) * m;
        for (int j = k + tid; j < m; j += bs) {
            double2 a = P[j];
            if (have_prev) {  // a -= v_k conj(w_j) + w_k conj(v_j)   (update of step k-1)
                const double2 vk = svp[k], wk = sw[k], vj = svp[j], wj = sw[j];
                a.x -= vk.x * wj.x + vk.y * wj.y + wk.x * vj.x + wk.y * vj.y;
                a.y -= vk.y * wj.x - vk.x * wj.y + wk.y * vj.x - wk.x * vj.y;
            }
            sr[j] = a;
        }
        __syncthreads();
        // reflector of the column below the diagonal, x_j = conj(r_j), j > k
        double part = 0.0;
        for (int j = k + 2 + tid; j < m; j += bs) part += sr[j].x * sr[j].x + sr[j].y * sr[j].y;
        const double xn2 = block_sum2(make_double2(part, 0.0), red).x;
        if (tid == 0) {  // the reflector's scalars once per CTA (FP64 divisions are costly)
            const double2 alpha = make_double2(sr[k + 1].x, -sr[k + 1].y);
            double2 t = make_double2(0.0, 0.0), scale = make_double2(0.0, 0.0);
            double beta = alpha.x;
            if (xn2 > 0.0 || alpha.y != 0.0) {
                beta = -copysign(sqrt(alpha.x * alpha.x + alpha.y * alpha.y + xn2), alpha.x);
                t = make_double2((beta - alpha.x) / beta, -alpha.y / beta);
                const double2 den = make_double2(alpha.x - beta, alpha.y);
                const double dd = den.x * den.x + den.y * den.y;
                scale = make_double2(den.x / dd, -den.y / dd);
            }
            s_sc[0] = t;
            s_sc[1] = scale;
            s_sc[2] = make_double2(beta, 0.0);
        }
        __syncthreads();
        const double2 t = s_sc[0], scale = s_sc[1];
        const double beta = s_sc[2].x;
        for (int j = k + 1 + tid; j < m; j += bs) {
            const double2 v = j == k + 1 ? make_double2(1.0, 0.0) : cmul(make_double2(sr[j].x, -sr[j].y), scale);
            sv[j] = v;
            if (b == 0) Vh[(size_t)k * m + j] = v;
        }
        if (b == 0 && tid == 0) {
            tau[k] = t;
            e[k] = beta;
            d[k] = sr[k].x;
        }
        __syncthreads();
        // 2. own rows i > k, 8 at a time: update of step k-1 (columns > k), then
        //    w_k[i] = t (A22 v_k)_i.  The threads stride over the columns (every warp busy on
        //    every row); the owner of row k+1 publishes its updated entries.
        const int r_first = k + 1 > b ? (k + 1 - b + G - 1) / G : 0;
        double2* pub = prow + (size_t)((k + 1) & 1) * m;
        for (int r0 = r_first; r0 < nr; r0 += 8) {
            const int rn = min(8, nr - r0);
            double2 acc[8], vi[8], wi[8];
            double2* rowp[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                acc[q] = make_double2(0.0, 0.0);
                const int i = b + G * (r0 + (q < rn ? q : 0));
                vi[q] = have_prev ? svp[i] : make_double2(0.0, 0.0);
                wi[q] = have_prev ? sw[i] : make_double2(0.0, 0.0);
                rowp[q] = kSmemRows ? srows + (size_t)(r0 + (q < rn ? q : 0)) * m : A + (size_t)i * lda;
            }
            const int q_pub = (k + 1 - b) % G == 0 ? (k + 1 - b) / G - r0 : -1;  // row k+1 in this chunk
            for (int j = k + 1 + tid; j < m; j += bs) {
                const double2 v = sv[j];
                const double2 vj = have_prev ? svp[j] : make_double2(0.0, 0.0);
                const double2 wj = have_prev ? sw[j] : make_double2(0.0, 0.0);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (q < rn) {
                        double2 a = rowp[q][j];
                        if (have_prev) {
                            a.x -= vi[q].x * wj.x + vi[q].y * wj.y + wi[q].x * vj.x + wi[q].y * vj.y;
                            a.y -= vi[q].y * wj.x - vi[q].x * wj.y + wi[q].y * vj.x - wi[q].x * vj.y;
                            rowp[q][j] = a;
                        }
                        if (q == q_pub) pub[j] = a;
                        acc[q].x += a.x * v.x - a.y * v.y;
                        acc[q].y += a.x * v.y + a.y * v.x;
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                if (q < rn) {
                    for (int o = 16; o > 0; o >>= 1) {
                        acc[q].x += __shfl_xor_sync(0xffffffffu, acc[q].x, o);
                        acc[q].y += __shfl_xor_sync(0xffffffffu, acc[q].y, o);
                    }
                    if (lane == 0) s_part[warp][q] = acc[q];
                }
            }
            __syncthreads();
            if (tid < rn) {
                double2 sum = make_double2(0.0, 0.0);
                for (int w8 = 0; w8 < 8; ++w8) {  // fixed order
                    sum.x += s_part[w8][tid].x;
                    sum.y += s_part[w8][tid].y;
                }
                wbuf[(size_t)(k & 1) * m + b + G * (r0 + tid)] = cmul(t, sum);
            }
            __syncthreads();
        }
        grid.sync();
        // 4. w_k with the symmetric correction; (v_k, w_k) become the previous update
        double2 dp = make_double2(0.0, 0.0);
        for (int j = k + 1 + tid; j < m; j += bs) {
            const double2 wj = wbuf[(size_t)(k & 1) * m + j];
            sw[j] = wj;
            const double2 c = cmulc(wj, sv[j]);
            dp.x += c.x;
            dp.y += c.y;
        }
        dp = block_sum2(dp, red);
        const double2 a2 = cmul(make_double2(-0.5 * t.x, -0.5 * t.y), dp);
        for (int j = k + 1 + tid; j < m; j += bs) {
            const double2 v = sv[j], av = cmul(a2, v);
            sw[j].x += av.x;
            sw[j].y += av.y;
            svp[j] = v;
        }
        __syncthreads();
        have_prev = true;
    }
    if (b == 0 && tid == 0) {
        double2 a = m == 1 ? A[0] : prow[(size_t)((m - 1) & 1) * m + (m - 1)];
        if (have_prev) {
            const double2 v = svp[m - 1], w = sw[m - 1];
            a.x -= 2.0 * (v.x * w.x + v.y * w.y);
        }
        d[m - 1] = a.x;
    }
}

// number of eigenvalues of T smaller than x (Sturm sequence with a pivot guard)
__device__ __forceinline__ int sturm_count(const double* __restrict__ d, const double* __restrict__ e2, int m,
                                           double x, double pivmin) {
    int c = 0;
    double q = d[0] - x;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0.0) ++c;
    for (int i = 1; i < m; ++i) {
        q = (d[i] - x) - e2[i - 1] / q;
        if (fabs(q) < pivmin) q = -pivmin;
        if (q < 0.0) ++c;
    }
    return c;
}

__global__ void k_sq(const double* __restrict__ e, double* __restrict__ e2, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) e2[i] = e[i] * e[i];
}

// one warp per wanted eigenvalue j < nev
__global__ void k_multisect(const double* __restrict__ d, const double* __restrict__ e, const double* __restrict__ e2,
                            int m, int nev, double* __restrict__ evals) {
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= nev) return;
    // Gershgorin interval and pivot guard
    double lo = 1e300, hi = -1e300, emax = 0.0;
    for (int i = lane; i < m; i += 32) {
        const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < m - 1 ? fabs(e[i]) : 0.0);
        lo = fmin(lo, d[i] - r);
        hi = fmax(hi, d[i] + r);
        if (i < m - 1) emax = fmax(emax, e2[i]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    }
    const double span = fmax(hi - lo, 1e-300);
    lo -= 1e-14 * span + 1e-300;
    hi += 1e-14 * span + 1e-300;
    const double pivmin = fmax(1e-300, 2.2250738585072014e-308 * fmax(1.0, emax));
    for (int round = 0; round < 14; ++round) {
        const double x = lo + (hi - lo) * (double)(lane + 1) / 33.0;
        const int c = sturm_count(d, e2, m, x, pivmin);
        const unsigned above = __ballot_sync(0xffffffffu, c > j);
        double nlo = lo, nhi = hi;
        if (above) {
            const int f = __ffs(above) - 1;
            nhi = __shfl_sync(0xffffffffu, x, f);
            if (f > 0) nlo = __shfl_sync(0xffffffffu, x, f - 1);
        } else {
            nlo = __shfl_sync(0xffffffffu, x, 31);
        }
        lo = nlo;
        hi = nhi;
        if (hi - lo <= 4.0e-16 * fmax(fabs(lo), fabs(hi)) + 1e-300) break;
    }
    if (lane == 0) evals[j] = 0.5 * (lo + hi);
}

// solve (T - lam) x = b in place (b -> x), T = tridiag(e, d, e); LU with partial pivoting.
// The row being eliminated is carried in registers (each finished row is stored once and only
// read back by the back substitution), so the loop has no read-after-write through memory.
// work: 3 arrays of m doubles (finished rows: pivot, first and second super-diagonal).
__device__ void tri_solve(const double* __restrict__ d, const double* __restrict__ e, int m, double lam,
                          double tiny, double* __restrict__ a, double* __restrict__ c, double* __restrict__ c2,
                          double* __restrict__ b) {
    // current row i: diag ai, super ci (and super-super c2i = 0 unless a swap put it there), rhs bi
    double ai = d[0] - lam, ci = (m > 1) ? e[0] : 0.0, bi = b[0];
    for (int i = 0; i < m - 1; ++i) {
        const double sub = e[i];
        // next original row i+1: sub, diag, sup, rhs
        double an = d[i + 1] - lam, cn = (i + 1 < m - 1) ? e[i + 1] : 0.0, bn = b[i + 1];
        double c2i = 0.0;
        if (fabs(ai) >= fabs(sub)) {
            if (ai == 0.0) ai = tiny;
            const double f = sub / ai;
            an -= f * ci;
            bn -= f * bi;
        } else {  // swap rows i and i+1
            const double f = ai / sub;
            const double ai0 = ai, ci0 = ci, bi0 = bi;
            ai = sub;
            ci = an;
            c2i = cn;
            bi = bn;
            an = ci0 - f * an;
            cn = -f * cn;
            bn = bi0 - f * bn;
            (void)ai0;
        }
        a[i] = ai;
        c[i] = ci;
        c2[i] = c2i;
        b[i] = bi;
        ai = an;
        ci = cn;
        bi = bn;
    }
    if (ai == 0.0) ai = tiny;
    a[m - 1] = ai;
    double x1 = bi / ai, x2 = 0.0;  // x[i+1], x[i+2]
    b[m - 1] = x1;
    for (int i = m - 2; i >= 0; --i) {
        const double xi = (b[i] - c[i] * x1 - c2[i] * x2) / a[i];
        b[i] = xi;
        x2 = x1;
        x1 = xi;
    }
}

// infinity norm of T and the cluster tolerance: eigenvalues closer than ctol form a cluster whose
// vectors are orthogonalised explicitly; outside clusters inverse iteration alone leaves a
// non-orthogonality of about eps * |T| / gap <= 1e-11
__device__ double tri_ctol(const double* __restrict__ d, const double* __restrict__ e, int m) {
    double tn = 0.0;
    for (int i = threadIdx.x & 31; i < m; i += 32)
        tn = fmax(tn, fabs(d[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < m - 1 ? fabs(e[i]) : 0.0));
    for (int o = 16; o > 0; o >>= 1) tn = fmax(tn, __shfl_xor_sync(0xffffffffu, tn, o));
    return tn;
}

// one warp per eigenvalue j: lane 0 runs the (sequential) tridiagonal solves of three inverse
// iterations from a deterministic start, the warp shares the O(m) vector work; the normalised
// vector is left in x_j = work + (4 j + 3) m.  Vectors of one cluster are orthogonalised
// afterwards (k_cluster_orth), so every eigenvalue's iterations run in parallel.
__global__ void __launch_bounds__(32)
k_inviter(const double* __restrict__ d, const double* __restrict__ e, int m, int nev,
          const double* __restrict__ evals, double* __restrict__ work) {
    const int j = blockIdx.x, lane = threadIdx.x;
    if (j >= nev) return;
    const double tn = tri_ctol(d, e, m);
    double* a = work + (size_t)j * 4 * m;
    double* c = a + m;
    double* c2 = c + m;
    double* x = c2 + m;
    const double tiny = 2.2e-16 * fmax(tn, 1e-200);
    const double lam = evals[j];
    // deterministic pseudo-random start (a counter hash of (j, i))
    for (int i = lane; i < m; i += 32) {
        unsigned h = 2654435761u * (unsigned)(j + 1) ^ (2246822519u * (unsigned)(i + 1));
        h ^= h >> 15;
        h *= 2246822519u;
        h ^= h >> 13;
        x[i] = ((double)(h >> 8) / 16777216.0) - 0.5;
    }
    __syncwarp();
    for (int it = 0; it < 3; ++it) {
        if (lane == 0) tri_solve(d, e, m, lam, tiny, a, c, c2, x);
        __syncwarp();
        double xm = 0.0;  // rescale before any sum of squares can overflow
        for (int i = lane; i < m; i += 32) xm = fmax(xm, fabs(x[i]));
        for (int o = 16; o > 0; o >>= 1) xm = fmax(xm, __shfl_xor_sync(0xffffffffu, xm, o));
        const double r = (xm > 0.0 && xm < 1e300) ? 1.0 / xm : 1.0;
        double nrm = 0.0;
        for (int i = lane; i < m; i += 32) {
            x[i] *= r;
            nrm += x[i] * x[i];
        }
        for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
        nrm = 1.0 / sqrt(nrm);
        for (int i = lane; i < m; i += 32) x[i] *= nrm;
        __syncwarp();
    }
}

// One CTA per cluster leader (eigenvalue j0 not within ctol of j0-1): the cluster's vectors
// j0..j1-1 are orthonormalised in order by two classical Gram-Schmidt passes against the
// earlier ones (dot products split over the warps), then written as columns of Y (imag 0).
__global__ void __launch_bounds__(256)
k_cluster_orth(const double* __restrict__ d, const double* __restrict__ e, int m, int nev,
               const double* __restrict__ evals, double* __restrict__ work, double2* __restrict__ Y, int ldy) {
    __shared__ double dots[256];
    __shared__ double red[32];
    const int j0 = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (j0 >= nev) return;
    const double ctol = 1e-5 * tri_ctol(d, e, m);  // every warp computes the same value
    if (j0 > 0 && evals[j0] - evals[j0 - 1] <= ctol) return;  // not a cluster leader
    int j1 = j0 + 1;
    while (j1 < nev && evals[j1] - evals[j1 - 1] <= ctol) ++j1;
    auto X = [&](int q) { return work + ((size_t)q * 4 + 3) * m; };
    for (int j = j0 + 1; j < j1; ++j) {
        double* x = X(j);
        for (int pass = 0; pass < 2; ++pass) {
            for (int q0 = j0; q0 < j; q0 += 256) {  // coefficients against up to 256 earlier vectors
                const int nq = min(256, j - q0);
                for (int q = warp; q < nq; q += 8) {
                    const double* y = X(q0 + q);
                    double s = 0.0;
                    for (int i = lane; i < m; i += 32) s += y[i] * x[i];
                    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                    if (lane == 0) dots[q] = s;
                }
                __syncthreads();
                for (int i = tid; i < m; i += 256) {
                    double v = x[i];
                    for (int q = 0; q < nq; ++q) v -= dots[q] * X(q0 + q)[i];
                    x[i] = v;
                }
                __syncthreads();
            }
        }
        double s = 0.0;
        for (int i = tid; i < m; i += 256) s += x[i] * x[i];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[warp] = s;
        __syncthreads();
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        const double inv = 1.0 / sqrt(t);
        for (int i = tid; i < m; i += 256) x[i] *= inv;
        __syncthreads();
    }
    for (int j = j0; j < j1; ++j)
        for (int i = tid; i < m; i += 256) Y[(size_t)i * ldy + j] = make_double2(X(j)[i], 0.0);
}

// y <- H_0 H_1 ... H_{m-2} y for column j of Y (one CTA per column)
__global__ void __launch_bounds__(256)
k_backtransf(const double2* __restrict__ Vh, const double2* __restrict__ tau, int m, double2* __restrict__ Y, int ldy) {
    extern __shared__ double2 sy[];
    __shared__ double2 red[32];
    const int j = blockIdx.x, tid = threadIdx.x, bs = blockDim.x;
    for (int i = tid; i < m; i += bs) sy[i] = Y[(size_t)i * ldy + j];
    __syncthreads();
    for (int k = m - 2; k >= 0; --k) {
        const double2 t = tau[k];
        if (t.x == 0.0 && t.y == 0.0) continue;
        const int n = m - k - 1;
        const double2* v = Vh + (size_t)k * m + (k + 1);
        double2 sp = make_double2(0.0, 0.0);
        for (int i = tid; i < n; i += bs) {
            const double2 c = cmulc(v[i], sy[k + 1 + i]);
            sp.x += c.x;
            sp.y += c.y;
        }
        const double2 s = cmul(t, block_sum2(sp, red));
        for (int i = tid; i < n; i += bs) {
            const double2 c = cmul(v[i], s);
            sy[k + 1 + i].x -= c.x;
            sy[k + 1 + i].y -= c.y;
        }
        __syncthreads();
    }
    for (int i = tid; i < m; i += bs) Y[(size_t)i * ldy + j] = sy[i];
}

}  // namespace

size_t heev_work_bytes(int m, int nev) {
    size_t b = 0;
    b += align_up((size_t)m * m * sizeof(double2), 256);      // Vh
    b += align_up((size_t)m * sizeof(double2), 256);          // tau
    b += align_up((size_t)2 * m * sizeof(double2), 256) * 2;  // wbuf, published rows (double-buffered)
    b += align_up((size_t)m * sizeof(double), 256) * 3;       // d, e, e2
    b += align_up((size_t)nev * 4 * m * sizeof(double), 256); // inverse-iteration scratch
    return b;
}

// Lowest nev eigenpairs of the Hermitian m x m matrix A (lda; destroyed).  evals: nev
// doubles (device, increasing); Y: m x nev (device, row-major, ld ldy) eigenvectors as columns.
// the process-wide stream of a device for cooperative launches (created on first use)
static qm_status cooperative_stream(int dev, cudaStream_t* out) {
    static std::mutex mu;
    static std::map<int, cudaStream_t> streams;
    std::lock_guard<std::mutex> lk(mu);
    auto it = streams.find(dev);
    if (it == streams.end()) {
        cudaStream_t cs = nullptr;
        qm_status st = cuda_check(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "cooperative stream");
        if (st) return st;
        it = streams.emplace(dev, cs).first;
    }
    *out = it->second;
    return QM_OK;
}

qm_status heev_lowest(double2* A, int lda, int m, int nev, double* evals, double2* Y, int ldy, void* work,
                      cudaStream_t s) {
    if (m <= 0 || nev <= 0) return QM_OK;
    if (nev > m) return fail(QM_ERR_ARG, "heev_lowest: nev > m");
    char* w = (char*)work;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* p = w + off;
        off += align_up(bytes, 256);
        return p;
    };
    double2* Vh = (double2*)take((size_t)m * m * sizeof(double2));
    double2* tau = (double2*)take((size_t)m * sizeof(double2));
    double2* wbuf = (double2*)take((size_t)2 * m * sizeof(double2));
    double2* prow = (double2*)take((size_t)2 * m * sizeof(double2));
    double* d = (double*)take((size_t)m * sizeof(double));
    double* e = (double*)take((size_t)m * sizeof(double));
    double* e2 = (double*)take((size_t)m * sizeof(double));
    double* iw = (double*)take((size_t)nev * 4 * m * sizeof(double));
    qm_status st;
    if (m == 1) {
        // T = (a11): copy the real diagonal, eigenvector 1
        cudaMemcpy2DAsync(evals, sizeof(double), A, sizeof(double2), sizeof(double), 1, cudaMemcpyDeviceToDevice, s);
        const double2 one = make_double2(1.0, 0.0);
        cudaMemcpyAsync(Y, &one, sizeof(double2), cudaMemcpyHostToDevice, s);
        return cuda_check(cudaGetLastError(), "heev m=1");
    }
    {
        int dev = 0, sms = 152;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        // one-barrier reduction: one CTA per SM (the FP64 work of a column is spread over the
        // whole GPU); rows in shared memory when they fit, else updated in place in A.  Beyond
        // 4 m vectors of shared memory, the two-barrier kernel (shared memory for 2 vectors only).
        const int G = std::max(1, std::min(sms, m));
        const size_t vec = 4 * (size_t)m * sizeof(double2);
        const size_t rows = (size_t)((m + G - 1) / G) * m * sizeof(double2);
        const void* kern = nullptr;
        size_t smem = 0;
        int blocks = G;
        if (vec + rows <= 200 * 1024) {
            kern = (const void*)k_tridiag_rows<true>;
            smem = vec + rows;
        } else if (vec <= 200 * 1024) {
            kern = (const void*)k_tridiag_rows<false>;
            smem = vec;
        } else {
            kern = (const void*)k_tridiag;
            smem = 2 * (size_t)m * sizeof(double2);
            if (smem > 200 * 1024) return fail(QM_ERR_UNSUPPORTED, "heev_lowest: m too large for the reduction kernel");
        }
        if ((st = allow_dynamic_smem(kern, smem, "heev_lowest: reduction kernel"))) return st;
        int occ = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, smem);
        if (occ < 1) return fail(QM_ERR_UNSUPPORTED, "heev_lowest: reduction kernel does not fit an SM");
        if (kern == (const void*)k_tridiag)  // fewer CTAs: two barriers per column
            blocks = std::min(std::min(occ * sms, std::max(1, (m + 7) / 8)), 64);
        blocks = std::min(blocks, occ * sms);
        if (kern != (const void*)k_tridiag && blocks != G)
            return fail(QM_ERR_UNSUPPORTED, "heev_lowest: reduction grid not resident");
        void* args_old[] = {(void*)&A, (void*)&lda, (void*)&m, (void*)&Vh, (void*)&tau, (void*)&d, (void*)&e,
                            (void*)&wbuf};
        void* args_new[] = {(void*)&A, (void*)&lda, (void*)&m, (void*)&Vh, (void*)&tau, (void*)&d, (void*)&e,
                            (void*)&wbuf, (void*)&prow};
        void** args = kern == (const void*)k_tridiag ? args_old : args_new;
        // Cooperative grids of concurrent callers (other host threads, other streams) must not
        // be resident at the same time: two partly resident grids could each wait at a grid
        // barrier for CTAs the other holds.  Every cooperative launch therefore goes through
        // one stream per device, joined to the caller's stream by events.
        cudaStream_t cs = nullptr;
        if ((st = cooperative_stream(dev, &cs))) return st;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if ((st = cuda_check(cudaEventCreateWithFlags(&e0, cudaEventDisableTiming), "event")) ||
            (st = cuda_check(cudaEventCreateWithFlags(&e1, cudaEventDisableTiming), "event")))
            return st;
        st = cuda_check(cudaEventRecord(e0, s), "event record");
        if (!st) st = cuda_check(cudaStreamWaitEvent(cs, e0, 0), "cooperative stream wait");
        if (!st) {
            ProfScope pf(PF_TRIDIAG, cs);
            st = cuda_check(cudaLaunchCooperativeKernel(kern, dim3(blocks), dim3(256), args, smem, cs),
                            "k_tridiag cooperative launch");
        }
        if (!st) st = cuda_check(cudaEventRecord(e1, cs), "event record");
        if (!st) st = cuda_check(cudaStreamWaitEvent(s, e1, 0), "stream wait");
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (st) return st;
    }
    {
        ProfScope pf(PF_MULTISECT, s);
        k_sq<<<(m + 255) / 256, 256, 0, s>>>(e, e2, m - 1);
    }
    {
        ProfScope pf(PF_MULTISECT, s);
        k_multisect<<<nev, 32, 0, s>>>(d, e, e2, m, nev, evals);
    }
    {
        ProfScope pf(PF_INVITER, s);
        k_inviter<<<nev, 32, 0, s>>>(d, e, m, nev, evals, iw);
    }
    {
        ProfScope pf(PF_INVITER, s);
        k_cluster_orth<<<nev, 256, 0, s>>>(d, e, m, nev, evals, iw, Y, ldy);
    }
    {
        const size_t smem = (size_t)m * sizeof(double2);
        if ((st = allow_dynamic_smem((const void*)k_backtransf, smem, "heev_lowest: back-transformation"))) return st;
        ProfScope pf(PF_BACKTR, s);
        k_backtransf<<<nev, 256, smem, s>>>(Vh, tau, m, Y, ldy);
    }
    return cuda_check(cudaGetLastError(), "heev launches");
}

}  // namespace qm

using namespace qm;

extern "C" qm_status qm_eigh_lowest(int m, int nev, const void* A, int lda, double* evals, void* Y, int ldy,
                                    void* stream) {
    clear_error();
    if (m <= 0 || nev <= 0 || nev > m) return fail(QM_ERR_ARG, "qm_eigh_lowest: need 0 < nev <= m");
    if (!A || !evals || !Y || lda < m || ldy < nev) return fail(QM_ERR_ARG, "qm_eigh_lowest: bad pointer or ld");
    if ((uintptr_t)A % 16 || (uintptr_t)Y % 16) return fail(QM_ERR_ARG, "qm_eigh_lowest: A, Y not 16-byte aligned");
    if (2 * (size_t)m * sizeof(double2) > 200 * 1024) return fail(QM_ERR_UNSUPPORTED, "qm_eigh_lowest: m > 6400");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t a_bytes = align_up((size_t)m * m * sizeof(double2), 256);
    void* work = nullptr;
    qm_status st = cuda_check(cudaMallocAsync(&work, a_bytes + heev_work_bytes(m, nev), s), "qm_eigh_lowest alloc");
    if (st) return st;
    double2* Aw = (double2*)work;
    st = cuda_check(cudaMemcpy2DAsync(Aw, (size_t)m * sizeof(double2), A, (size_t)lda * sizeof(double2),
                                      (size_t)m * sizeof(double2), m, cudaMemcpyDeviceToDevice, s),
                    "qm_eigh_lowest copy");
    if (!st) st = heev_lowest(Aw, m, m, nev, evals, (double2*)Y, ldy, (char*)work + a_bytes, s);
    cudaFreeAsync(work, s);
    return st;
}
