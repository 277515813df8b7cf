// Lowest eigenpairs of a complex Hermitian matrix in FP64, for the Rayleigh-Ritz step of the
// Davidson solver (and the Loewdin orthonormalisation).  Classical dense algorithms, written
// for a GPU whose FP64 rate is low: the O(m^3) work is done once (Householder reduction), and
// only the wanted eigenpairs are computed from the tridiagonal matrix.
//
//   1. k_tridiag      Householder reduction Q^H A Q = T, T real symmetric tridiagonal
//                     (Golub & Van Loan, Matrix Computations, Sec. 8.3.1; the complex
//                     reflector makes every subdiagonal element real).  One cooperative
//                     launch; two grid barriers per column.
//   2. k_multisect    the j-th smallest eigenvalue of T by multisection on Sturm counts
//                     (Sec. 8.4.1): a warp tests 32 points per round, 12 rounds.
//   3. k_inviter      eigenvectors of T by inverse iteration (LU with partial pivoting of the
//                     tridiagonal, three solves), Gram-Schmidt within clusters of close
//                     eigenvalues (Sec. 8.4.2, 8.2.2).
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

// one warp per cluster leader: lane 0 runs the (sequential) tridiagonal solves, the warp
// shares the O(m) vector work (start vector, Gram-Schmidt within the cluster, scaling).
// Eigenvector j of T -> Y[i*ldy + j] (complex, imag 0).
__global__ void __launch_bounds__(32)
k_inviter(const double* __restrict__ d, const double* __restrict__ e, int m, int nev,
          const double* __restrict__ evals, double* __restrict__ work, double2* __restrict__ Y, int ldy) {
    const int j0 = blockIdx.x, lane = threadIdx.x;
    if (j0 >= nev) return;
    double tn = 0.0;  // infinity norm of T
    for (int i = lane; i < m; i += 32)
        tn = fmax(tn, fabs(d[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < m - 1 ? fabs(e[i]) : 0.0));
    for (int o = 16; o > 0; o >>= 1) tn = fmax(tn, __shfl_xor_sync(0xffffffffu, tn, o));
    // eigenvalues closer than ctol form a cluster whose vectors are orthogonalised explicitly;
    // outside clusters inverse iteration alone leaves a non-orthogonality of about
    // eps * |T| / gap <= 1e-11
    const double ctol = 1e-5 * tn;
    if (j0 > 0 && evals[j0] - evals[j0 - 1] <= ctol) return;  // not a cluster leader
    int j1 = j0 + 1;
    while (j1 < nev && evals[j1] - evals[j1 - 1] <= ctol) ++j1;
    double* a = work + (size_t)j0 * 4 * m;
    double* c = a + m;
    double* c2 = c + m;
    double* x = c2 + m;
    const double tiny = 2.2e-16 * fmax(tn, 1e-200);
    for (int j = j0; j < j1; ++j) {
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
            for (int i = lane; i < m; i += 32) x[i] *= r;
            __syncwarp();
            for (int q = j0; q < j; ++q) {  // orthogonalise against the cluster's earlier vectors
                double dot = 0.0;
                for (int i = lane; i < m; i += 32) dot += Y[(size_t)i * ldy + q].x * x[i];
                for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
                for (int i = lane; i < m; i += 32) x[i] -= dot * Y[(size_t)i * ldy + q].x;
                __syncwarp();
            }
            double nrm = 0.0;
            for (int i = lane; i < m; i += 32) nrm += x[i] * x[i];
            for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
            nrm = 1.0 / sqrt(nrm);
            for (int i = lane; i < m; i += 32) x[i] *= nrm;
            __syncwarp();
        }
        for (int i = lane; i < m; i += 32) Y[(size_t)i * ldy + j] = make_double2(x[i], 0.0);
        __syncwarp();
    }
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
    b += align_up((size_t)m * sizeof(double2), 256) * 2;      // tau, wbuf
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
    double2* wbuf = (double2*)take((size_t)m * sizeof(double2));
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
        const size_t smem = 2 * (size_t)m * sizeof(double2);
        if (smem > 200 * 1024) return fail(QM_ERR_UNSUPPORTED, "heev_lowest: m too large for the reduction kernel");
        if ((st = allow_dynamic_smem((const void*)k_tridiag, smem, "heev_lowest: reduction kernel"))) return st;
        int dev = 0, sms = 152, occ = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_tridiag, 256, smem);
        // fewer CTAs than SMs: the FP64 work per column is small and grid barriers get cheaper
        int blocks = std::max(1, std::min(std::max(1, occ) * sms, std::max(1, (m + 7) / 8)));
        blocks = std::min(blocks, 64);
        void* args[] = {(void*)&A, (void*)&lda, (void*)&m, (void*)&Vh, (void*)&tau, (void*)&d, (void*)&e,
                        (void*)&wbuf};
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
            st = cuda_check(cudaLaunchCooperativeKernel((void*)k_tridiag, dim3(blocks), dim3(256), args, smem, cs),
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
        k_inviter<<<nev, 32, 0, s>>>(d, e, m, nev, evals, iw, Y, ldy);
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
