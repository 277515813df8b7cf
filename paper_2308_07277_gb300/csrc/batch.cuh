// Batched H psi over many independent (cell, k-point) jobs in ONE persistent launch.
//
// Every job is the operator of qm_hpsi (Eq. KSHamMat with the KB term of Sec. 2.3, local
// part by the IFFT / V(r) / FFT recipe of Sec. 4.3, stick-pruned as in Sec. 4.3.3).  The
// work of all jobs is cut into items of seven kinds, listed in one array in phase order:
//
//   VT   (cell, chunk)          V(r)/N_r in the permuted plane order of the FFT path
//   NLP  (job, chunk, block)    partial projections <beta_p|psi_b> over a chunk of plane waves
//   K1   (job, tile)            scatter + inverse x transform of a tile of (band, stick) lines
//   NLR  (job)                  reduce the partials in a fixed order: Pd[b][p] = D_p <beta_p|psi_b>
//   K2   (job, band group, p1)  y/z inverse transforms, V multiply, z/y forward transforms of
//                               one yz plane for a group of bands (planes stacked in shared memory)
//   K3   (job, tile)            forward x transform, gather, + 1/2|k+G|^2 psi
//   NLA  (job, G tile)          out += sum_p beta_p Pd[b][p]
//
// CTAs take items with a global ticket counter (atomicAdd; a CTA holds its current ticket and
// the next one), so items start in array order.
// An item waits (thread 0 polls a per-job counter with acquire loads) only for items of an
// earlier phase, which hold smaller tickets and are therefore already running on resident
// CTAs: the scheme cannot deadlock whatever the grid size.  A finished item publishes its
// writes with a fence and a counter increment.  Data produced inside the launch is read
// with ld.global.cg (L2), never through the non-coherent or L1 paths.  Every wait is bounded;
// on expiry the CTA sets the error word and the remaining waits give up at once.
#pragma once
#include "fft_kernels.cuh"

namespace qm {

enum BatchKind : int { BK_VT = 0, BK_NLP, BK_K1, BK_NLR, BK_K2, BK_K3, BK_NLA, kBatchKinds };
enum BatchCounter : int { BC_K1 = 0, BC_K2, BC_K3, BC_NLP, BC_NLR, kBatchCounters = 8 };

constexpr int kBatchSG = 32;           // plane waves per projection sub-step
constexpr int kBatchGA = 64;           // plane waves per application item
constexpr int kBatchGC = 512;          // plane waves per projection chunk
constexpr int kBatchVTC = 8192;        // V(r) elements per layout item
constexpr int kBatchAB = 48;           // bands per application pass (12 per thread)
constexpr int kBatchAP = 16;           // projectors per staged block of Pd
constexpr long long kBatchSpinLimit = 1ll << 24;

// One job; pointers are device pointers, element types follow the launch's precision.
struct BatchJobDev {
    int n1, n2, n3, ldx, ldy;
    int nstick, nstick_pad, nrow, npw, nb, nproj;
    int nl, nk1;      // (band, stick) lines per stick item; stick items per phase
    int bpp, nk2;     // bands per plane item; plane items
    int nchunk;       // projection chunks of kBatchGC plane waves
    int bblk, nbblk;  // bands per projection item; band blocks
    int nnla;         // application items
    int cell;
    int pad_;
    long long ld_psi, ld_out, ld_beta;
    AxisPlan px, py, pz;
    const int* stick_g0;
    const int* stick_plane;
    const int2* g_code;
    const void* kin;
    const int* rows2;  // [bpp * nrow] stacked plane rows: (l / nrow) * N3 + rows[l % nrow]
    const int* cols2;  // [bpp * N2] stacked plane columns: (l / N2) * N3 * ldy + l % N2
    const void* tw[3];
    const void* psi;
    void* out;
    const void* beta;
    const double* D;
    void* T;     // [nb][N1][nstick_pad] stick buffer
    void* part;  // [nchunk][nb][nproj] partial projections
    void* Pd;    // [nb][nproj]
};

struct BatchCellDev {
    const double* V;
    void* vt;
    int n1, n2, n3, nchunk;
    const int* rev[3];
    double scale;
};

// Host-written controls of the bounded waits (device memory, read at every item, so that the
// captured graph need not change): the poll limit of every wait, and a failure-detection test
// hook that makes the last-phase (K3) items of one job wait for one completion more than will
// ever arrive.
struct BatchCtl {
    long long spin_limit;  // polls per bounded wait
    int hold_job;          // job whose K3 waits need hold_extra more plane items (-1: none)
    int hold_extra;
};

struct BatchLaunch {
    const BatchCtl* ctl;
    const BatchJobDev* jobs;
    const BatchCellDev* cells;
    const int4* items;
    int nitems;
    int* cnt;       // [njobs * kBatchCounters]
    int* cell_cnt;  // [ncells]
    int* head;      // ticket counter
    int* err;       // error word
    int order;      // radix order of the FFT plans (0 or 1)
    int grid;
    size_t smem;
};

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed_gpu(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// bounded wait for *p >= target; false on expiry (sets *err) or when *err is already set
__device__ __forceinline__ bool batch_wait(const int* p, int target, int* err, long long limit) {
    for (long long it = 0; it < limit; ++it) {
        if (ld_acquire_gpu(p) >= target) return true;
        if (ld_relaxed_gpu(err)) return false;
        __nanosleep(64);
    }
    atomicExch(err, 1);
    return false;
}

template <class C> __device__ __forceinline__ C ldcg(const C* p);
template <> __device__ __forceinline__ float2 ldcg(const float2* p) { return __ldcg(p); }
template <> __device__ __forceinline__ double2 ldcg(const double2* p) { return __ldcg(p); }
template <> __device__ __forceinline__ float ldcg(const float* p) { return __ldcg(p); }
template <> __device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }

// The FFT lengths of the batched workload get compile-time plans; others take the runtime plan.
#define QM_FFT_LENGTHS_BATCH(X) X(18) X(20) X(24) X(25) X(27) X(30) X(32) X(36) X(40) X(45) X(48) X(50) X(54) X(60) X(64)

// ORD: radix order of the compile-time plans (0: large radices first, 1: reversed); the
// job's runtime AxisPlans and the cells' digit-reversal tables follow the same order.
template <class C, int SG, bool DIF, bool LINE_FAST, int ORD>
__device__ void fft_lines_b(C* buf, int es, int ls, int nlines, const int* lmap, const AxisPlan& pl, const C* tw,
                            int tid, int nt) {
    switch (pl.n) {
#define QM_CASE(n) \
    case n: fft_lines_ct<C, SG, DIF, LINE_FAST, n, ORD>(buf, es, ls, nlines, lmap, tw, tid, nt); return;
        QM_FFT_LENGTHS_BATCH(QM_CASE)
#undef QM_CASE
        default: break;
    }
    if (DIF) {
        for (int s = 0; s < pl.nst; ++s) {
            fft_stage_any<C, SG, DIF, LINE_FAST>(pl.r[s], buf, es, ls, nlines, lmap, pl.L[s], pl.n, tw, tid, nt);
            __syncthreads();
        }
    } else {
        for (int s = pl.nst - 1; s >= 0; --s) {
            fft_stage_any<C, SG, DIF, LINE_FAST>(pl.r[s], buf, es, ls, nlines, lmap, pl.L[s], pl.n, tw, tid, nt);
            __syncthreads();
        }
    }
}

// z transforms of stacked planes with the V multiply between them (see fft_z_vmul_ct)
template <class C, class R, int ORD>
__device__ void fft_z_vmul_b(C* buf, int ldy, int ncol, const int* cmap, int nv, const R* __restrict__ v, int ldv,
                             const AxisPlan& pz, const C* tw, int tid, int nt) {
    switch (pz.n) {
#define QM_CASE(n) \
    case n: fft_z_vmul_ct<C, R, n, ORD>(buf, ldy, ncol, cmap, nv, v, ldv, tw, tid, nt); return;
        QM_FFT_LENGTHS_BATCH(QM_CASE)
#undef QM_CASE
        default: break;
    }
    fft_lines_b<C, +1, true, true, ORD>(buf, ldy, 1, ncol, cmap, pz, tw, tid, nt);
    for (int i = tid; i < pz.n * ncol; i += nt) {
        const int r = i / ncol, l = i - r * ncol;
        const R sc = __ldcg(v + r * ldv + l % nv);
        C* x = buf + (cmap ? cmap[l] : l) + r * ldy;
        const C y = *x;
        *x = mk<C>(y.x * sc, y.y * sc);
    }
    __syncthreads();
    fft_lines_b<C, -1, false, true, ORD>(buf, ldy, 1, ncol, cmap, pz, tw, tid, nt);
}

// ---------------------------------------------------------------- item bodies
template <class R>
__device__ void bk_vt(const BatchCellDev& c, int chunk, int tid, int nt) {
    const int N1 = c.n1, N2 = c.n2, N3 = c.n3;
    const long long nr = (long long)N1 * N2 * N3;
    const long long i0 = (long long)chunk * kBatchVTC;
    const long long i1 = i0 + kBatchVTC < nr ? i0 + kBatchVTC : nr;
    R* vt = (R*)c.vt;
    for (long long i = i0 + tid; i < i1; i += nt) {
        const int p2 = (int)(i % N2);
        const long long q = i / N2;
        const int p3 = (int)(q % N3);
        const int p1 = (int)(q / N3);
        const long long src = (long long)__ldg(c.rev[0] + p1) +
                              (long long)N1 * ((long long)__ldg(c.rev[1] + p2) + (long long)N2 * __ldg(c.rev[2] + p3));
        vt[i] = (R)(__ldg(c.V + src) * c.scale);
    }
}

// K1: lines [L0, L1) of the job's (band, stick) list, line L = b * nstick + s
template <class R, int ORD>
__device__ void bk_k1(const BatchJobDev& J, int tile, unsigned char* sm, int tid, int nt) {
    using C = typename Cx<R>::T;
    const int N1 = J.n1, ldx = J.ldx, nst = J.nstick;
    const int L0 = tile * J.nl;
    const int L1 = min(L0 + J.nl, J.nb * nst);
    const int nlines = L1 - L0;
    C* lines = (C*)sm;
    C* tw = lines + (size_t)J.nl * ldx;
    const C* twg = (const C*)J.tw[0];
    for (int i = tid; i < N1; i += nt) tw[i] = twg[i];
    for (int i = tid; i < nlines * ldx; i += nt) lines[i] = mk<C>(0, 0);
    __syncthreads();
    const C* psi = (const C*)J.psi;
    for (int L = L0; L < L1;) {
        const int b = L / nst, sa = L - b * nst;
        const int sb = min(nst, sa + (L1 - L));
        const int gb = __ldg(J.stick_g0 + sa), ge = __ldg(J.stick_g0 + sb);
        const C* src = psi + (size_t)b * J.ld_psi;
        const int base = b * nst - L0;
        for (int g = gb + tid; g < ge; g += nt) {
            const int2 c = __ldg(J.g_code + g);
            lines[(base + c.x) * ldx + c.y] = src[g];
        }
        L += sb - sa;
    }
    __syncthreads();
    fft_lines_b<C, +1, true, false, ORD>(lines, 1, ldx, nlines, nullptr, J.px, tw, tid, nt);
    C* T = (C*)J.T;
    const RDiv dl{nlines, 1.0f / (float)nlines};
    for (int i = tid; i < N1 * nlines; i += nt) {
        const int p = dl.div(i), l = i - p * nlines;
        const int L = L0 + l, b = L / nst, s = L - b * nst;
        T[((size_t)b * N1 + p) * J.nstick_pad + s] = lines[l * ldx + p];
    }
}

// K2: plane p1 of bands [b0, b0 + nbp), the planes stacked in shared memory
template <class R, int ORD>
__device__ void bk_k2(const BatchJobDev& J, const R* vt, int grp, int p1, unsigned char* sm, int tid, int nt) {
    using C = typename Cx<R>::T;
    const int N1 = J.n1, N2 = J.n2, N3 = J.n3, ldy = J.ldy, nst = J.nstick;
    const int b0 = grp * J.bpp;
    const int nbp = min(J.bpp, J.nb - b0);
    const int ps = N3 * ldy;
    C* plane = (C*)sm;
    C* twy = plane + (size_t)J.bpp * ps;
    C* twz = twy + N2;
    const C* twgy = (const C*)J.tw[1];
    const C* twgz = (const C*)J.tw[2];
    for (int i = tid; i < N2; i += nt) twy[i] = twgy[i];
    for (int i = tid; i < N3; i += nt) twz[i] = twgz[i];
    for (int i = tid; i < nbp * ps; i += nt) plane[i] = mk<C>(0, 0);
    __syncthreads();
    C* T = (C*)J.T;
    const RDiv ds{nst, 1.0f / (float)nst};
    for (int i = tid; i < nbp * nst; i += nt) {
        const int bi = ds.div(i), s = i - bi * nst;
        plane[bi * ps + __ldg(J.stick_plane + s)] = ldcg(T + ((size_t)(b0 + bi) * N1 + p1) * J.nstick_pad + s);
    }
    __syncthreads();
    fft_lines_b<C, +1, true, false, ORD>(plane, 1, ldy, nbp * J.nrow, J.rows2, J.py, twy, tid, nt);
    // z: inverse, V(r)/N_r, forward (one fused pass for the compile-time lengths)
    fft_z_vmul_b<C, R, ORD>(plane, ldy, nbp * N2, J.cols2, N2, vt + (size_t)p1 * N3 * N2, N2, J.pz, twz, tid, nt);
    fft_lines_b<C, -1, false, false, ORD>(plane, 1, ldy, nbp * J.nrow, J.rows2, J.py, twy, tid, nt);
    for (int i = tid; i < nbp * nst; i += nt) {
        const int bi = ds.div(i), s = i - bi * nst;
        T[((size_t)(b0 + bi) * N1 + p1) * J.nstick_pad + s] = plane[bi * ps + __ldg(J.stick_plane + s)];
    }
}

// K3: forward x transform of lines [L0, L1), gather the sphere, add the kinetic term
template <class R, int ORD>
__device__ void bk_k3(const BatchJobDev& J, int tile, unsigned char* sm, int tid, int nt) {
    using C = typename Cx<R>::T;
    const int N1 = J.n1, ldx = J.ldx, nst = J.nstick;
    const int L0 = tile * J.nl;
    const int L1 = min(L0 + J.nl, J.nb * nst);
    const int nlines = L1 - L0;
    C* lines = (C*)sm;
    C* tw = lines + (size_t)J.nl * ldx;
    const C* twg = (const C*)J.tw[0];
    for (int i = tid; i < N1; i += nt) tw[i] = twg[i];
    const C* T = (const C*)J.T;
    const RDiv dl{nlines, 1.0f / (float)nlines};
    for (int i = tid; i < N1 * nlines; i += nt) {
        const int p = dl.div(i), l = i - p * nlines;
        const int L = L0 + l, b = L / nst, s = L - b * nst;
        lines[l * ldx + p] = ldcg(T + ((size_t)b * N1 + p) * J.nstick_pad + s);
    }
    __syncthreads();
    fft_lines_b<C, -1, false, false, ORD>(lines, 1, ldx, nlines, nullptr, J.px, tw, tid, nt);
    const C* psi = (const C*)J.psi;
    C* out = (C*)J.out;
    const R* kin = (const R*)J.kin;
    for (int L = L0; L < L1;) {
        const int b = L / nst, sa = L - b * nst;
        const int sb = min(nst, sa + (L1 - L));
        const int gb = __ldg(J.stick_g0 + sa), ge = __ldg(J.stick_g0 + sb);
        const C* ps = psi + (size_t)b * J.ld_psi;
        C* po = out + (size_t)b * J.ld_out;
        const int base = b * nst - L0;
        for (int g = gb + tid; g < ge; g += nt) {
            const int2 c = __ldg(J.g_code + g);
            const C x = lines[(base + c.x) * ldx + c.y];
            const C y = ps[g];
            const R k = __ldg(kin + g);
            po[g] = mk<C>(x.x + k * y.x, x.y + k * y.y);
        }
        L += sb - sa;
    }
}

// NLP: part[chunk][b][p] = sum_{G in chunk} conj(beta_p(G)) psi_b(G), bands of block `blk`;
// each active thread owns a 4 x 4 (band x projector) register tile
template <class R>
__device__ void bk_nlp(const BatchJobDev& J, int chunk, int blk, unsigned char* sm, int tid, int nt) {
    using C = typename Cx<R>::T;
    const int np = J.nproj;
    const int g0 = chunk * kBatchGC, g1 = min(J.npw, g0 + kBatchGC);
    const int b0 = blk * J.bblk, nbk = min(J.bblk, J.nb - b0);
    const int nbt = (nbk + 3) >> 2, npt = (np + 3) >> 2;
    const int npad = npt * 4, bpad = nbt * 4;
    C* sb = (C*)sm;               // [kBatchSG][npad]
    C* sp = sb + kBatchSG * npad;  // [kBatchSG][4][nbt]: band 4 bt + i at [q][i][bt] (conflict-free reads)
    const C* beta = (const C*)J.beta;
    const C* psi = (const C*)J.psi;
    const bool active = tid < nbt * npt;
    const int bt = active ? tid % nbt : 0, pt = active ? tid / nbt : 0;
    C acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = mk<C>(0, 0);
    for (int gs = g0; gs < g1; gs += kBatchSG) {
        const int ng = min(kBatchSG, g1 - gs);
        for (int i = tid; i < npad * kBatchSG; i += nt) {
            const int p = i / kBatchSG, q = i - p * kBatchSG;
            sb[q * npad + p] = (p < np && q < ng) ? beta[(size_t)p * J.ld_beta + gs + q] : mk<C>(0, 0);
        }
        for (int i = tid; i < bpad * kBatchSG; i += nt) {
            const int b = i / kBatchSG, q = i - b * kBatchSG;
            sp[q * bpad + (b & 3) * nbt + (b >> 2)] =
                (b < nbk && q < ng) ? psi[(size_t)(b0 + b) * J.ld_psi + gs + q] : mk<C>(0, 0);
        }
        __syncthreads();
        if (active) {
            for (int q = 0; q < ng; ++q) {
                C a[4], w[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = sp[q * bpad + i * nbt + bt];
#pragma unroll
                for (int j = 0; j < 4; ++j) w[j] = sb[q * npad + 4 * pt + j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        // conj(w) * a
                        acc[i][j].x += w[j].x * a[i].x + w[j].y * a[i].y;
                        acc[i][j].y += w[j].x * a[i].y - w[j].y * a[i].x;
                    }
            }
        }
        __syncthreads();
    }
    if (active) {
        C* part = (C*)J.part;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int b = 4 * bt + i;
            if (b >= nbk) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int p = 4 * pt + j;
                if (p < np) part[((size_t)chunk * J.nb + b0 + b) * np + p] = acc[i][j];
            }
        }
    }
}

// NLR: Pd[b][p] = D_p * sum_chunks part[c][b][p], chunks added in increasing order
template <class R>
__device__ void bk_nlr(const BatchJobDev& J, int tid, int nt) {
    using C = typename Cx<R>::T;
    const int np = J.nproj, nb = J.nb;
    const C* part = (const C*)J.part;
    C* Pd = (C*)J.Pd;
    for (int e = tid; e < nb * np; e += nt) {
        const int p = e % np;
        C s = mk<C>(0, 0);
        for (int c = 0; c < J.nchunk; ++c) {
            const C v = ldcg(part + (size_t)c * nb * np + e);
            s.x += v.x;
            s.y += v.y;
        }
        const R d = (R)__ldg(J.D + p);
        Pd[e] = mk<C>(s.x * d, s.y * d);
    }
}

// NLA: out[b][G] += sum_p beta_p(G) Pd[b][p] for the plane waves of one tile; thread
// (G = tid % 64, h = tid / 64) accumulates bands h, h + 4, ... (12 per pass)
template <class R>
__device__ void bk_nla(const BatchJobDev& J, int tile, unsigned char* sm, int tid, int nt) {
    using C = typename Cx<R>::T;
    const int np = J.nproj, nb = J.nb;
    const int g = tile * kBatchGA + (tid & (kBatchGA - 1));
    const int h = tid / kBatchGA;
    const bool gv = g < J.npw && h < 4;
    const C* beta = (const C*)J.beta;
    const C* Pd = (const C*)J.Pd;
    C* out = (C*)J.out;
    C* sPd = (C*)sm;  // [kBatchAB][kBatchAP]
    for (int b0 = 0; b0 < nb; b0 += kBatchAB) {
        const int nbk = min(kBatchAB, nb - b0);
        C acc[kBatchAB / 4];
#pragma unroll
        for (int i = 0; i < kBatchAB / 4; ++i) acc[i] = mk<C>(0, 0);
        for (int p0 = 0; p0 < np; p0 += kBatchAP) {
            const int npk = min(kBatchAP, np - p0);
            __syncthreads();
            for (int i = tid; i < kBatchAB * kBatchAP; i += nt) {
                const int b = i / kBatchAP, p = i - b * kBatchAP;
                sPd[i] = (b < nbk && p < npk) ? ldcg(Pd + (size_t)(b0 + b) * np + p0 + p) : mk<C>(0, 0);
            }
            __syncthreads();
            if (gv) {
                for (int p = 0; p < npk; ++p) {
                    const C w = __ldg(beta + (size_t)(p0 + p) * J.ld_beta + g);
#pragma unroll
                    for (int i = 0; i < kBatchAB / 4; ++i) {
                        const C d = sPd[(h + 4 * i) * kBatchAP + p];
                        acc[i].x += w.x * d.x - w.y * d.y;
                        acc[i].y += w.x * d.y + w.y * d.x;
                    }
                }
            }
        }
        if (gv) {
#pragma unroll
            for (int i = 0; i < kBatchAB / 4; ++i) {
                const int b = h + 4 * i;
                if (b < nbk) {
                    C* o = out + (size_t)(b0 + b) * J.ld_out + g;
                    const C x = ldcg(o);
                    *o = mk<C>(x.x + acc[i].x, x.y + acc[i].y);
                }
            }
        }
    }
}

// ---------------------------------------------------------------- the persistent kernel
template <class R, int ORD>
__global__ void __launch_bounds__(kThreads, sizeof(R) == 4 ? 3 : 2)  // FP32: 3 CTAs per SM, FP64: 2
k_batch(const BatchCtl* __restrict__ ctl, const BatchJobDev* __restrict__ jobs, const BatchCellDev* __restrict__ cells,
        const int4* __restrict__ items, int nitems, int* cnt, int* cell_cnt, int* head, int* err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(16) BatchJobDev J;
    __shared__ int s_item, s_next, s_go;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) s_item = atomicAdd(head, 1);
    __syncthreads();
    for (;;) {
        const int it = s_item;
        if (it >= nitems) return;
        // the next ticket is taken now (its latency hides behind this item); it is larger than
        // this one, so every wait still points to a smaller ticket than the waiter's
        if (tid == 0) s_next = atomicAdd(head, 1);
        const int4 w = __ldg(items + it);
        if (w.x != BK_VT) {
            const int* src = reinterpret_cast<const int*>(jobs + w.y);
            int* dst = reinterpret_cast<int*>(&J);
            for (int i = tid; i < (int)(sizeof(BatchJobDev) / sizeof(int)); i += nt) dst[i] = __ldg(src + i);
        }
        if (tid == 0) {
            bool go = true;
            const int* c = cnt + (size_t)w.y * kBatchCounters;
            const long long lim = ctl->spin_limit;
            switch (w.x) {
                case BK_NLR: go = batch_wait(c + BC_NLP, jobs[w.y].nchunk * jobs[w.y].nbblk, err, lim); break;
                case BK_K2: {
                    const int cell = jobs[w.y].cell;
                    go = batch_wait(c + BC_K1, jobs[w.y].nk1, err, lim) &&
                         batch_wait(cell_cnt + cell, cells[cell].nchunk, err, lim);
                    break;
                }
                case BK_K3:
                    go = batch_wait(c + BC_K2, jobs[w.y].nk2 + (w.y == ctl->hold_job ? ctl->hold_extra : 0), err, lim);
                    break;
                case BK_NLA:
                    go = batch_wait(c + BC_K3, jobs[w.y].nk1, err, lim) && batch_wait(c + BC_NLR, 1, err, lim);
                    break;
                default: break;
            }
            if (go) __threadfence();
            s_go = go ? 1 : 0;
        }
        __syncthreads();
        if (s_go) {
            switch (w.x) {
                case BK_VT: bk_vt<R>(cells[w.y], w.z, tid, nt); break;
                case BK_NLP: bk_nlp<R>(J, w.z, w.w, smem_raw, tid, nt); break;
                case BK_K1: bk_k1<R, ORD>(J, w.z, smem_raw, tid, nt); break;
                case BK_NLR: bk_nlr<R>(J, tid, nt); break;
                case BK_K2: bk_k2<R, ORD>(J, (const R*)cells[J.cell].vt, w.z, w.w, smem_raw, tid, nt); break;
                case BK_K3: bk_k3<R, ORD>(J, w.z, smem_raw, tid, nt); break;
                case BK_NLA: bk_nla<R>(J, w.z, smem_raw, tid, nt); break;
                default: break;
            }
        }
        __syncthreads();
        if (tid == 0) {
            int* c = nullptr;
            switch (w.x) {
                case BK_VT: c = cell_cnt + w.y; break;
                case BK_NLP: c = cnt + (size_t)w.y * kBatchCounters + BC_NLP; break;
                case BK_K1: c = cnt + (size_t)w.y * kBatchCounters + BC_K1; break;
                case BK_NLR: c = cnt + (size_t)w.y * kBatchCounters + BC_NLR; break;
                case BK_K2: c = cnt + (size_t)w.y * kBatchCounters + BC_K2; break;
                case BK_K3: c = cnt + (size_t)w.y * kBatchCounters + BC_K3; break;
                default: break;
            }
            if (c) {
                __threadfence();
                atomicAdd(c, 1);
            }
            s_item = s_next;
        }
        __syncthreads();
    }
}

// batch_occupancy_impl raises the kernel's dynamic shared memory limit to the per-CTA
// maximum (the attribute is per function, and graphs of several batches hold different sizes).
template <class R>
qm_status batch_launch_impl(const BatchLaunch& L, cudaStream_t s) {
    if (L.order)
        k_batch<R, 1><<<L.grid, kThreads, L.smem, s>>>(L.ctl, L.jobs, L.cells, L.items, L.nitems, L.cnt, L.cell_cnt,
                                                       L.head, L.err);
    else
        k_batch<R, 0><<<L.grid, kThreads, L.smem, s>>>(L.ctl, L.jobs, L.cells, L.items, L.nitems, L.cnt, L.cell_cnt,
                                                       L.head, L.err);
    return cuda_check(cudaGetLastError(), "batched H psi launch");
}

// resident CTAs per SM at `smem` bytes of dynamic shared memory (0 if it does not fit)
template <class R, int ORD>
int batch_occupancy_ord(size_t smem) {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa{};
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, k_batch<R, ORD>) != cudaSuccess)
        return 0;
    const int max_dyn = optin - (int)fa.sharedSizeBytes;
    if ((long long)smem > max_dyn) return 0;
    if (cudaFuncSetAttribute(k_batch<R, ORD>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch<R, ORD>, kThreads, smem) != cudaSuccess) return 0;
    return n;
}
template <class R>
int batch_occupancy_impl(size_t smem, int order) {
    return order ? batch_occupancy_ord<R, 1>(smem) : batch_occupancy_ord<R, 0>(smem);
}

}  // namespace qm
