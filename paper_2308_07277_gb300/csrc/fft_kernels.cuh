// Local-potential + kinetic part of H psi by stick-pruned 3D FFTs staged in shared memory.
//
// The operator is the recipe of Sec. 4.3 (IFFT of psi(G), multiply by V(r), FFT, keep the
// sphere) with the kinetic term 1/2|k+G|^2 applied in G-space (Sec. 4.3), and the stick
// pruning of Sec. 4.3.3: 1D transforms run only on lines that can hold non-zero data.
//
// Data flow for one band (x fastest on the grid, sticks along x as in the paper's Fig. 1):
//   K1 k_stick_inverse : scatter the sphere into the x-sticks that hold plane waves
//                        (zero fill), inverse FFT along x  -> stick buffer T[b][p1][s]
//   K2 k_plane         : one yz plane per (band, p1): expand sticks into the plane,
//                        inverse FFT along y (active rows only) and z, multiply by V(r)/N_r,
//                        forward FFT along z and y (active rows), compact back into T
//   K3 k_stick_forward : forward FFT along x, gather the sphere, add 1/2|k+G|^2 psi(G)
//
// Every 1D transform is an in-place mixed-radix (2/3/4/5/8/9) FFT in shared memory.  The
// inverse passes are decimation-in-frequency (natural order in, digit-reversed out) and the
// forward passes decimation-in-time (digit-reversed in, natural out), so the digit
// reversal never has to be undone: the only quantity that lives in the permuted order is
// V(r), which is laid out once per call in that order (k_vt).
#pragma once
#include <algorithm>

#include "qm_internal.h"

namespace qm {

template <class R> struct Cx;
template <> struct Cx<double> { using T = double2; };
template <> struct Cx<float> { using T = float2; };

template <class C> __device__ __forceinline__ C mk(decltype(C::x) a, decltype(C::x) b) {
    C r;
    r.x = a;
    r.y = b;
    return r;
}
template <class C> __device__ __forceinline__ C add(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <class C> __device__ __forceinline__ C sub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <class C> __device__ __forceinline__ C cmul(C a, C w) {
    return mk<C>(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
}
// multiply by SG * i
template <class C, int SG> __device__ __forceinline__ C mul_si(C a) {
    return SG > 0 ? mk<C>(-a.y, a.x) : mk<C>(a.y, -a.x);
}
template <class C, int SG> __device__ __forceinline__ C twid(const C* tw, int t) {
    C w = tw[t];
    if (SG < 0) w.y = -w.y;
    return w;
}

// In-register DFT of length R with kernel exp(SG * 2 pi i n k / R).
template <class C, int SG, int R> struct Dft;

template <class C, int SG> struct Dft<C, SG, 2> {
    static __device__ __forceinline__ void run(C* u) {
        C a = u[0], b = u[1];
        u[0] = add(a, b);
        u[1] = sub(a, b);
    }
};
template <class C, int SG> struct Dft<C, SG, 4> {
    static __device__ __forceinline__ void run(C* u) {
        C a = add(u[0], u[2]), b = sub(u[0], u[2]);
        C c = add(u[1], u[3]), d = mul_si<C, SG>(sub(u[1], u[3]));
        u[0] = add(a, c);
        u[2] = sub(a, c);
        u[1] = add(b, d);
        u[3] = sub(b, d);
    }
};
template <class C, int SG> struct Dft<C, SG, 3> {
    static __device__ __forceinline__ void run(C* u) {
        using R = decltype(C::x);
        const R h = (R)0.86602540378443864676;  // sin(2 pi / 3)
        C t = add(u[1], u[2]);
        C d = mul_si<C, SG>(sub(u[1], u[2]));
        C m = mk<C>(u[0].x - (R)0.5 * t.x, u[0].y - (R)0.5 * t.y);
        u[0] = add(u[0], t);
        u[1] = mk<C>(m.x + h * d.x, m.y + h * d.y);
        u[2] = mk<C>(m.x - h * d.x, m.y - h * d.y);
    }
};
template <class C, int SG> struct Dft<C, SG, 5> {
    static __device__ __forceinline__ void run(C* u) {
        using R = decltype(C::x);
        const R c1 = (R)0.30901699437494742410;   // cos(2 pi / 5)
        const R c2 = (R)-0.80901699437494742410;  // cos(4 pi / 5)
        const R s1 = (R)0.95105651629515357212;   // sin(2 pi / 5)
        const R s2 = (R)0.58778525229247312917;   // sin(4 pi / 5)
        C t1 = add(u[1], u[4]), t2 = add(u[2], u[3]);
        C d1 = mul_si<C, SG>(sub(u[1], u[4])), d2 = mul_si<C, SG>(sub(u[2], u[3]));
        C a1 = mk<C>(u[0].x + c1 * t1.x + c2 * t2.x, u[0].y + c1 * t1.y + c2 * t2.y);
        C a2 = mk<C>(u[0].x + c2 * t1.x + c1 * t2.x, u[0].y + c2 * t1.y + c1 * t2.y);
        C b1 = mk<C>(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y);
        C b2 = mk<C>(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y);
        u[0] = add(u[0], add(t1, t2));
        u[1] = add(a1, b1);
        u[4] = sub(a1, b1);
        u[2] = add(a2, b2);
        u[3] = sub(a2, b2);
    }
};

template <class C, int SG> struct Dft<C, SG, 8> {
    // 8 = 2 x 4: two 4-point DFTs on the even and odd inputs, combined with w8^k
    static __device__ __forceinline__ void run(C* u) {
        using R = decltype(C::x);
        C a[4] = {u[0], u[2], u[4], u[6]}, b[4] = {u[1], u[3], u[5], u[7]};
        Dft<C, SG, 4>::run(a);
        Dft<C, SG, 4>::run(b);
        const R h = (R)0.70710678118654752440;  // 1/sqrt(2)
        const C w1 = mk<C>(h * b[1].x - (R)SG * h * b[1].y, h * b[1].y + (R)SG * h * b[1].x);  // (1+SG i)/sqrt2 b1
        const C w2 = mul_si<C, SG>(b[2]);                                                         // SG i b2
        const C w3 = mk<C>(-h * b[3].x - (R)SG * h * b[3].y, -h * b[3].y + (R)SG * h * b[3].x);  // (-1+SG i)/sqrt2 b3
        u[0] = add(a[0], b[0]);
        u[4] = sub(a[0], b[0]);
        u[1] = add(a[1], w1);
        u[5] = sub(a[1], w1);
        u[2] = add(a[2], w2);
        u[6] = sub(a[2], w2);
        u[3] = add(a[3], w3);
        u[7] = sub(a[3], w3);
    }
};
template <class C, int SG> struct Dft<C, SG, 9> {
    // 9 = 3 x 3: 3-point DFTs over the stride-3 subsequences, twiddles w9^(j k1), 3-point
    // DFTs across them; output index k1 + 3 k2
    static __device__ __forceinline__ void run(C* u) {
        using R = decltype(C::x);
        const R c1 = (R)0.76604444311897803520, s1 = (R)0.64278760968653932632;   // 2 pi / 9
        const R c2 = (R)0.17364817766693034885, s2 = (R)0.98480775301220805936;   // 4 pi / 9
        const R c4 = (R)-0.93969262078590838405, s4 = (R)0.34202014332566873304;  // 8 pi / 9
        C a0[3] = {u[0], u[3], u[6]}, a1[3] = {u[1], u[4], u[7]}, a2[3] = {u[2], u[5], u[8]};
        Dft<C, SG, 3>::run(a0);
        Dft<C, SG, 3>::run(a1);
        Dft<C, SG, 3>::run(a2);
        a1[1] = cmul(a1[1], mk<C>(c1, (R)SG * s1));
        a1[2] = cmul(a1[2], mk<C>(c2, (R)SG * s2));
        a2[1] = cmul(a2[1], mk<C>(c2, (R)SG * s2));
        a2[2] = cmul(a2[2], mk<C>(c4, (R)SG * s4));
#pragma unroll
        for (int k1 = 0; k1 < 3; ++k1) {
            C col[3] = {a0[k1], a1[k1], a2[k1]};
            Dft<C, SG, 3>::run(col);
            u[k1] = col[0];
            u[k1 + 3] = col[1];
            u[k1 + 6] = col[2];
        }
    }
};

// One in-place stage over `nlines` lines of length N.  Element j of line l is
// buf[lmap(l) * ls + j * es].  DIF: butterfly then twiddle; DIT: twiddle then butterfly.
// LINE_FAST maps consecutive threads to consecutive lines (column passes), otherwise to
// consecutive butterflies of one line (row passes).
template <class C, int SG, int R, bool DIF, bool LINE_FAST>
__device__ __forceinline__ void fft_stage(C* buf, int es, int ls, int nlines, const int* lmap,
                                          int L, int N, const C* tw, int tid, int nt) {
    const int M = L / R;
    const int nbf = N / R;
    const int step = N / L;
    const int total = nlines * nbf;
    for (int t = tid; t < total; t += nt) {
        int line, bf;
        if (LINE_FAST) {
            line = t % nlines;
            bf = t / nlines;
        } else {
            line = t / nbf;
            bf = t - line * nbf;
        }
        const int blk = bf / M;
        const int n1 = bf - blk * M;
        const int lrow = lmap ? lmap[line] : line;  // the map may live in shared memory
        C* p = buf + lrow * ls + (blk * L + n1) * es;
        const int me = M * es;
        C u[R];
#pragma unroll
        for (int j = 0; j < R; ++j) u[j] = p[j * me];
        if (DIF) {
            Dft<C, SG, R>::run(u);
#pragma unroll
            for (int k2 = 1; k2 < R; ++k2) u[k2] = cmul(u[k2], twid<C, SG>(tw, n1 * k2 * step));
        } else {
#pragma unroll
            for (int k2 = 1; k2 < R; ++k2) u[k2] = cmul(u[k2], twid<C, SG>(tw, n1 * k2 * step));
            Dft<C, SG, R>::run(u);
        }
#pragma unroll
        for (int j = 0; j < R; ++j) p[j * me] = u[j];
    }
}

template <class C, int SG, bool DIF, bool LINE_FAST>
__device__ __forceinline__ void fft_stage_any(int r, C* buf, int es, int ls, int nlines, const int* lmap,
                                              int L, int N, const C* tw, int tid, int nt) {
    switch (r) {
        case 2: fft_stage<C, SG, 2, DIF, LINE_FAST>(buf, es, ls, nlines, lmap, L, N, tw, tid, nt); break;
        case 3: fft_stage<C, SG, 3, DIF, LINE_FAST>(buf, es, ls, nlines, lmap, L, N, tw, tid, nt); break;
        case 4: fft_stage<C, SG, 4, DIF, LINE_FAST>(buf, es, ls, nlines, lmap, L, N, tw, tid, nt); break;
        case 8: fft_stage<C, SG, 8, DIF, LINE_FAST>(buf, es, ls, nlines, lmap, L, N, tw, tid, nt); break;
        case 9: fft_stage<C, SG, 9, DIF, LINE_FAST>(buf, es, ls, nlines, lmap, L, N, tw, tid, nt); break;
        default: fft_stage<C, SG, 5, DIF, LINE_FAST>(buf, es, ls, nlines, lmap, L, N, tw, tid, nt); break;
    }
}

// ---------------------------------------------------------------- compile-time lengths
// For the common lengths the radix plan is a compile-time constant, so every stage's block
// length, butterfly count and twiddle step are constants and the per-butterfly index
// arithmetic reduces to multiply/shift (the runtime-radix stages above spend most of their
// instructions on integer division).  Same plan as the host's make_plan: 8s, then at most one
// 4 and one 2, 9s, at most one 3, 5s (few stages = few passes through shared memory).
struct CPlan {
    int nst;
    int r[kMaxStages];
    int L[kMaxStages];
};
// ord = 0: that radix sequence; ord = 1: the same radices in reverse order (small radices first;
// the batched form's autotuner chooses between the two, see fft_plan in gspace.cpp)
constexpr CPlan make_cplan(int n, int ord = 0) {
    int rs[kMaxStages] = {}, nr = 0, m = n;
    while (m % 8 == 0) { rs[nr++] = 8; m /= 8; }
    if (m % 4 == 0) { rs[nr++] = 4; m /= 4; }
    if (m % 2 == 0) { rs[nr++] = 2; m /= 2; }
    while (m % 9 == 0) { rs[nr++] = 9; m /= 9; }
    if (m % 3 == 0) { rs[nr++] = 3; m /= 3; }
    while (m % 5 == 0) { rs[nr++] = 5; m /= 5; }
    CPlan p{};
    int L = n;
    for (int i = 0; i < nr; ++i) {
        const int r = ord ? rs[nr - 1 - i] : rs[i];
        p.r[p.nst] = r;
        p.L[p.nst] = L;
        ++p.nst;
        L /= r;
    }
    return p;
}

// t / d for the runtime divisor d (t < 2^24): float reciprocal plus one correction step
struct RDiv {
    int d;
    float inv;
    __device__ __forceinline__ int div(int t) const {
        int q = __float2int_rz((float)t * inv);
        q += (q + 1) * d <= t;
        q -= q * d > t;
        return q;
    }
};

template <class C, int SG, int R, int L, int N, bool DIF, bool LINE_FAST>
__device__ __forceinline__ void fft_stage_ct(C* buf, int es, int ls, int nlines, RDiv ld, const int* lmap,
                                             const C* tw, int tid, int nt) {
    constexpr int M = L / R;
    constexpr int NBF = N / R;
    constexpr int STEP = N / L;
    const int total = nlines * NBF;
    for (int t = tid; t < total; t += nt) {
        int line, bf;
        if (LINE_FAST) {
            bf = ld.div(t);
            line = t - bf * nlines;
        } else {
            line = t / NBF;
            bf = t - line * NBF;
        }
        const int blk = bf / M;
        const int n1 = bf - blk * M;
        const int lrow = lmap ? lmap[line] : line;  // the map may live in shared memory
        C* p = buf + lrow * ls + (blk * L + n1) * es;
        const int me = M * es;
        C u[R];
#pragma unroll
        for (int j = 0; j < R; ++j) u[j] = p[j * me];
        // a stage with one butterfly per block (M = 1) has unit twiddles: no multiply (exact)
        if (DIF) {
            Dft<C, SG, R>::run(u);
            if constexpr (M > 1) {
#pragma unroll
                for (int k2 = 1; k2 < R; ++k2) u[k2] = cmul(u[k2], twid<C, SG>(tw, n1 * k2 * STEP));
            }
        } else {
            if constexpr (M > 1) {
#pragma unroll
                for (int k2 = 1; k2 < R; ++k2) u[k2] = cmul(u[k2], twid<C, SG>(tw, n1 * k2 * STEP));
            }
            Dft<C, SG, R>::run(u);
        }
#pragma unroll
        for (int j = 0; j < R; ++j) p[j * me] = u[j];
    }
}

// stage S of the plan of N (DIF order), then the rest (DIF: S+1 .. ; DIT: S-1 .. 0)
template <class C, int SG, bool DIF, bool LINE_FAST, int N, int S, int ORD = 0>
__device__ __forceinline__ void fft_stages_ct(C* buf, int es, int ls, int nlines, RDiv ld, const int* lmap,
                                              const C* tw, int tid, int nt) {
    constexpr CPlan P = make_cplan(N, ORD);
    if constexpr (S >= 0 && S < P.nst) {
        fft_stage_ct<C, SG, P.r[S], P.L[S], N, DIF, LINE_FAST>(buf, es, ls, nlines, ld, lmap, tw, tid, nt);
        __syncthreads();
        fft_stages_ct<C, SG, DIF, LINE_FAST, N, DIF ? S + 1 : S - 1, ORD>(buf, es, ls, nlines, ld, lmap, tw, tid, nt);
    }
}

// stages S, S+1, ..., END-1 of the plan of N in DIF order
template <class C, int SG, bool LINE_FAST, int N, int S, int END, int ORD = 0>
__device__ __forceinline__ void fft_stages_ct_to(C* buf, int es, int ls, int nlines, RDiv ld, const int* lmap,
                                                 const C* tw, int tid, int nt) {
    constexpr CPlan P = make_cplan(N, ORD);
    if constexpr (S < END) {
        fft_stage_ct<C, SG, P.r[S], P.L[S], N, true, LINE_FAST>(buf, es, ls, nlines, ld, lmap, tw, tid, nt);
        __syncthreads();
        fft_stages_ct_to<C, SG, LINE_FAST, N, S + 1, END, ORD>(buf, es, ls, nlines, ld, lmap, tw, tid, nt);
    }
}

// Inverse z transform of the ncol columns of a plane (or of stacked planes: column l starts
// at cmap[l], NULL = l), multiplication by the real V, forward z transform.  The last DIF
// stage of the inverse and the first DIT stage of the forward transform act on the same
// blocks of consecutive z positions with unit twiddles, so they and the V multiply are one
// pass in registers (bitwise the same result as three passes).  V of element (z, column l) is
// v[z * ldv + l % nv] (nv = columns of one plane), read through L2 (it may have been written
// by the same launch).
template <class C, class R, int N, int ORD = 0>
__device__ __forceinline__ void fft_z_vmul_ct(C* buf, int ldy, int ncol, const int* cmap, int nv,
                                              const R* __restrict__ v, int ldv, const C* tw, int tid, int nt) {
    constexpr CPlan P = make_cplan(N, ORD);
    constexpr int RL = P.r[P.nst - 1];
    constexpr int NBLK = N / RL;
    RDiv ld{ncol, 1.0f / (float)ncol};
    RDiv dv{nv, 1.0f / (float)nv};
    fft_stages_ct_to<C, +1, true, N, 0, P.nst - 1, ORD>(buf, ldy, 1, ncol, ld, cmap, tw, tid, nt);
    for (int t = tid; t < ncol * NBLK; t += nt) {
        const int blk = ld.div(t);
        const int col = t - blk * ncol;
        const int vc = cmap ? col - dv.div(col) * nv : col;
        C* p = buf + (cmap ? cmap[col] : col) + blk * RL * ldy;
        const R* vv = v + vc + blk * RL * ldv;
        C u[RL];
#pragma unroll
        for (int j = 0; j < RL; ++j) u[j] = p[j * ldy];
        Dft<C, +1, RL>::run(u);
#pragma unroll
        for (int j = 0; j < RL; ++j) {
            const R sc = __ldcg(vv + j * ldv);  // L2 path: V may have been written by the same launch
            u[j] = mk<C>(u[j].x * sc, u[j].y * sc);
        }
        Dft<C, -1, RL>::run(u);
#pragma unroll
        for (int j = 0; j < RL; ++j) p[j * ldy] = u[j];
    }
    __syncthreads();
    fft_stages_ct<C, -1, false, true, N, P.nst - 2, ORD>(buf, ldy, 1, ncol, ld, cmap, tw, tid, nt);
}

template <class C, int SG, bool DIF, bool LINE_FAST, int N, int ORD = 0>
__device__ __forceinline__ void fft_lines_ct(C* buf, int es, int ls, int nlines, const int* lmap, const C* tw,
                                             int tid, int nt) {
    constexpr CPlan P = make_cplan(N, ORD);
    RDiv ld{nlines, 1.0f / (float)nlines};
    fft_stages_ct<C, SG, DIF, LINE_FAST, N, DIF ? 0 : P.nst - 1, ORD>(buf, es, ls, nlines, ld, lmap, tw, tid, nt);
}

#define QM_FFT_LENGTHS(X) \
    X(18) X(20) X(24) X(25) X(30) X(32) X(36) X(40) X(45) X(48) X(50) X(54) X(60) X(64) X(72) X(75) \
    X(80) X(90) X(96) X(100) X(108) X(120) X(125) X(128) X(144)

// Full 1D transform of `nlines` lines; ends with __syncthreads().
template <class C, int SG, bool DIF, bool LINE_FAST>
__device__ void fft_lines(C* buf, int es, int ls, int nlines, const int* lmap, const AxisPlan& pl,
                          const C* tw, int tid, int nt) {
    switch (pl.n) {
#define QM_CASE(n) \
    case n: fft_lines_ct<C, SG, DIF, LINE_FAST, n>(buf, es, ls, nlines, lmap, tw, tid, nt); return;
        QM_FFT_LENGTHS(QM_CASE)
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

// z transforms of a plane (or stacked planes, see fft_z_vmul_ct) with the V multiply between
// them (ends with __syncthreads())
template <class C, class R>
__device__ void fft_z_vmul(C* buf, int ldy, int ncol, const int* cmap, int nv, const R* __restrict__ v, int ldv,
                           const AxisPlan& pz, const C* tw, int tid, int nt) {
    switch (pz.n) {
#define QM_CASE(n) \
    case n: fft_z_vmul_ct<C, R, n>(buf, ldy, ncol, cmap, nv, v, ldv, tw, tid, nt); return;
        QM_FFT_LENGTHS(QM_CASE)
#undef QM_CASE
        default: break;
    }
    fft_lines<C, +1, true, true>(buf, ldy, 1, ncol, cmap, pz, tw, tid, nt);
    for (int i = tid; i < pz.n * ncol; i += nt) {
        const int r = i / ncol, l = i - r * ncol;
        const R sc = __ldcg(v + r * ldv + l % nv);
        C* x = buf + (cmap ? cmap[l] : l) + r * ldy;
        const C y = *x;
        *x = mk<C>(y.x * sc, y.y * sc);
    }
    __syncthreads();
    fft_lines<C, -1, false, true>(buf, ldy, 1, ncol, cmap, pz, tw, tid, nt);
}

// ---------------------------------------------------------------- two register passes per 1D FFT
// The stages of a compile-time plan are split after stage K: stages [0, K) act on strided groups
// of a line (the thread with offset n < MB holds x[n + m MB], m < N/MB, MB = L[K] = the block
// length of stage K) and stages [K, nst) on contiguous sub-blocks of MB elements.  Each group is
// loaded into registers once, all its stages run there, and it is stored once: two passes
// through shared memory per 1D transform instead of one per stage.  The butterflies, twiddles
// and their order are those of the one-stage-per-pass code above, so the results are identical
// (DIF: natural order in, digit-reversed out; DIT the reverse).  K minimises the larger group.
constexpr int fused_split(int n) {
    CPlan p = make_cplan(n);
    int best = p.nst, bestv = n;
    for (int k = 1; k <= p.nst; ++k) {
        const int mb = k < p.nst ? p.L[k] : 1;
        const int v = (n / mb > mb) ? n / mb : mb;
        if (v < bestv) {
            bestv = v;
            best = k;
        }
    }
    return best;
}
template <int N> struct Fused {
    static constexpr CPlan P = make_cplan(N);
    static constexpr int K = fused_split(N);
    static constexpr int MB = K < P.nst ? P.L[K] : 1;  // contiguous sub-block length
    static constexpr int NA = N / MB;                   // elements of a strided group
    // used where it saves passes (plans of three or more stages) and a group fits the register budget
    static constexpr bool ok = P.nst >= 3 && (NA > MB ? NA : MB) <= 18;
};

// stage S on a strided group u[m] = x[n + m MB] (S < K)
template <class C, int SG, bool DIF, int N, int S>
__device__ __forceinline__ void stage_strided(C* u, int n, const C* tw) {
    constexpr CPlan P = make_cplan(N);
    constexpr int MB = Fused<N>::MB;
    constexpr int R = P.r[S], L = P.L[S], M = L / R, STEP = N / L;
#pragma unroll
    for (int blk = 0; blk < N / L; ++blk) {
#pragma unroll
        for (int q = 0; q < M / MB; ++q) {
            C v[R];
#pragma unroll
            for (int j = 0; j < R; ++j) v[j] = u[blk * (L / MB) + q + j * (M / MB)];
            const int n1 = n + q * MB;
            if (DIF) {
                Dft<C, SG, R>::run(v);
                if constexpr (M > 1) {
#pragma unroll
                    for (int k2 = 1; k2 < R; ++k2) v[k2] = cmul(v[k2], twid<C, SG>(tw, n1 * k2 * STEP));
                }
            } else {
                if constexpr (M > 1) {
#pragma unroll
                    for (int k2 = 1; k2 < R; ++k2) v[k2] = cmul(v[k2], twid<C, SG>(tw, n1 * k2 * STEP));
                }
                Dft<C, SG, R>::run(v);
            }
#pragma unroll
            for (int j = 0; j < R; ++j) u[blk * (L / MB) + q + j * (M / MB)] = v[j];
        }
    }
}

// stage S on a contiguous sub-block u[i] = x[b MB + i] (S >= K): every index is a constant
template <class C, int SG, bool DIF, int N, int S>
__device__ __forceinline__ void stage_block(C* u, const C* tw) {
    constexpr CPlan P = make_cplan(N);
    constexpr int MB = Fused<N>::MB;
    constexpr int R = P.r[S], L = P.L[S], M = L / R, STEP = N / L;
#pragma unroll
    for (int blk = 0; blk < MB / L; ++blk) {
#pragma unroll
        for (int n1 = 0; n1 < M; ++n1) {
            C v[R];
#pragma unroll
            for (int j = 0; j < R; ++j) v[j] = u[blk * L + n1 + j * M];
            if (DIF) {
                Dft<C, SG, R>::run(v);
                if constexpr (M > 1) {
#pragma unroll
                    for (int k2 = 1; k2 < R; ++k2) v[k2] = cmul(v[k2], twid<C, SG>(tw, n1 * k2 * STEP));
                }
            } else {
                if constexpr (M > 1) {
#pragma unroll
                    for (int k2 = 1; k2 < R; ++k2) v[k2] = cmul(v[k2], twid<C, SG>(tw, n1 * k2 * STEP));
                }
                Dft<C, SG, R>::run(v);
            }
#pragma unroll
            for (int j = 0; j < R; ++j) u[blk * L + n1 + j * M] = v[j];
        }
    }
}

// stages of a group in plan order: DIF S = S0, S0+1, ..., S1-1; DIT S = S1-1, ..., S0
template <class C, int SG, bool DIF, int N, int S, int S1>
__device__ __forceinline__ void strided_stages(C* u, int n, const C* tw) {
    if constexpr (S < S1) {
        if constexpr (DIF) {
            stage_strided<C, SG, true, N, S>(u, n, tw);
            strided_stages<C, SG, true, N, S + 1, S1>(u, n, tw);
        } else {
            strided_stages<C, SG, false, N, S + 1, S1>(u, n, tw);
            stage_strided<C, SG, false, N, S>(u, n, tw);
        }
    }
}
template <class C, int SG, bool DIF, int N, int S, int S1>
__device__ __forceinline__ void block_stages(C* u, const C* tw) {
    if constexpr (S < S1) {
        if constexpr (DIF) {
            stage_block<C, SG, true, N, S>(u, tw);
            block_stages<C, SG, true, N, S + 1, S1>(u, tw);
        } else {
            block_stages<C, SG, false, N, S + 1, S1>(u, tw);
            stage_block<C, SG, false, N, S>(u, tw);
        }
    }
}

// item t of a pass over nlines lines with G groups each -> (line, group).  Consecutive threads
// take the same group of consecutive lines, so a warp's accesses step by the line stride: one
// element apart in column passes, an odd padded row length apart in row passes (ldx, ldy are
// odd), i.e. free of shared-memory bank conflicts either way; a thread's group itself (strided
// or contiguous) never shares a warp access with its neighbours' elements.
template <bool LINE_FAST>
__device__ __forceinline__ void item_of(int t, int nlines, int G, RDiv dl, int& line, int& grp) {
    (void)G;
    grp = dl.div(t);
    line = t - grp * nlines;
}

// pass over the strided groups of nlines lines (stages [0, K)); ends with __syncthreads()
template <class C, int SG, bool DIF, bool LINE_FAST, int N>
__device__ __forceinline__ void pass_strided(C* buf, int es, int ls, int nlines, const int* lmap, const C* tw, int tid,
                                             int nt) {
    using F = Fused<N>;
    RDiv dl{nlines, 1.0f / (float)nlines};
    for (int t = tid; t < nlines * F::MB; t += nt) {
        int line, n;
        item_of<LINE_FAST>(t, nlines, F::MB, dl, line, n);
        C* p = buf + (lmap ? lmap[line] : line) * ls + n * es;
        C u[F::NA];
#pragma unroll
        for (int m = 0; m < F::NA; ++m) u[m] = p[m * F::MB * es];
        strided_stages<C, SG, DIF, N, 0, F::K>(u, n, tw);
#pragma unroll
        for (int m = 0; m < F::NA; ++m) p[m * F::MB * es] = u[m];
    }
    __syncthreads();
}

// pass over the contiguous sub-blocks of nlines lines (stages [K, nst)); ends with __syncthreads()
template <class C, int SG, bool DIF, bool LINE_FAST, int N>
__device__ __forceinline__ void pass_block(C* buf, int es, int ls, int nlines, const int* lmap, const C* tw, int tid,
                                           int nt) {
    using F = Fused<N>;
    if constexpr (F::K < F::P.nst) {
        RDiv dl{nlines, 1.0f / (float)nlines};
        for (int t = tid; t < nlines * F::NA; t += nt) {
            int line, b;
            item_of<LINE_FAST>(t, nlines, F::NA, dl, line, b);
            C* p = buf + (lmap ? lmap[line] : line) * ls + b * F::MB * es;
            C u[F::MB];
#pragma unroll
            for (int i = 0; i < F::MB; ++i) u[i] = p[i * es];
            block_stages<C, SG, DIF, N, F::K, F::P.nst>(u, tw);
#pragma unroll
            for (int i = 0; i < F::MB; ++i) p[i * es] = u[i];
        }
        __syncthreads();
    }
}

// full 1D transform of nlines lines in two register passes; ends with __syncthreads()
template <class C, int SG, bool DIF, bool LINE_FAST, int N>
__device__ __forceinline__ void fft2_lines_ct(C* buf, int es, int ls, int nlines, const int* lmap, const C* tw,
                                              int tid, int nt) {
    if (DIF) {
        pass_strided<C, SG, true, LINE_FAST, N>(buf, es, ls, nlines, lmap, tw, tid, nt);
        pass_block<C, SG, true, LINE_FAST, N>(buf, es, ls, nlines, lmap, tw, tid, nt);
    } else {
        pass_block<C, SG, false, LINE_FAST, N>(buf, es, ls, nlines, lmap, tw, tid, nt);
        pass_strided<C, SG, false, LINE_FAST, N>(buf, es, ls, nlines, lmap, tw, tid, nt);
    }
}

// z transforms of the ncol columns of one plane (natural column order, column l at buf + l,
// element z at z * ldy) with the V multiply between the inverse and forward transforms:
// inverse strided pass, one register pass of [inverse inner stages, x V(z), forward inner
// stages] per sub-block, forward strided pass (a single register pass when the plan has no
// sub-blocks).  V of (z position p, column l) is v[p * ldv + l], read through L2.
template <class C, class R, int N>
__device__ __forceinline__ void fft2_z_vmul_ct(C* buf, int ldy, int ncol, const R* __restrict__ v, int ldv,
                                               const C* tw, int tid, int nt) {
    using F = Fused<N>;
    RDiv dl{ncol, 1.0f / (float)ncol};
    if constexpr (F::K < F::P.nst) {
        pass_strided<C, +1, true, true, N>(buf, ldy, 1, ncol, nullptr, tw, tid, nt);
        for (int t = tid; t < ncol * F::NA; t += nt) {
            int col, b;
            item_of<true>(t, ncol, F::NA, dl, col, b);
            C* p = buf + col + b * F::MB * ldy;
            const R* vv = v + col + b * F::MB * ldv;
            C u[F::MB];
#pragma unroll
            for (int i = 0; i < F::MB; ++i) u[i] = p[i * ldy];
            block_stages<C, +1, true, N, F::K, F::P.nst>(u, tw);
#pragma unroll
            for (int i = 0; i < F::MB; ++i) {
                const R sc = __ldcg(vv + i * ldv);
                u[i] = mk<C>(u[i].x * sc, u[i].y * sc);
            }
            block_stages<C, -1, false, N, F::K, F::P.nst>(u, tw);
#pragma unroll
            for (int i = 0; i < F::MB; ++i) p[i * ldy] = u[i];
        }
        __syncthreads();
        pass_strided<C, -1, false, true, N>(buf, ldy, 1, ncol, nullptr, tw, tid, nt);
    } else {  // one group holds the whole column
        for (int col = tid; col < ncol; col += nt) {
            C* p = buf + col;
            C u[N];
#pragma unroll
            for (int m = 0; m < N; ++m) u[m] = p[m * ldy];
            strided_stages<C, +1, true, N, 0, F::K>(u, 0, tw);
#pragma unroll
            for (int m = 0; m < N; ++m) {
                const R sc = __ldcg(v + col + m * ldv);
                u[m] = mk<C>(u[m].x * sc, u[m].y * sc);
            }
            strided_stages<C, -1, false, N, 0, F::K>(u, 0, tw);
#pragma unroll
            for (int m = 0; m < N; ++m) p[m * ldy] = u[m];
        }
        __syncthreads();
    }
}

// dispatch: two-pass register transforms for the lengths whose groups fit the register
// budget, the stage-per-pass code otherwise (both end with __syncthreads())
template <class C, int SG, bool DIF, bool LINE_FAST>
__device__ void fft2_lines(C* buf, int es, int ls, int nlines, const int* lmap, const AxisPlan& pl, const C* tw,
                           int tid, int nt) {
    switch (pl.n) {
#define QM_CASE(n)                                                                                \
    case n:                                                                                       \
        if constexpr (Fused<n>::ok) {                                                             \
            fft2_lines_ct<C, SG, DIF, LINE_FAST, n>(buf, es, ls, nlines, lmap, tw, tid, nt);      \
            return;                                                                               \
        }                                                                                         \
        break;
        QM_FFT_LENGTHS(QM_CASE)
#undef QM_CASE
        default: break;
    }
    fft_lines<C, SG, DIF, LINE_FAST>(buf, es, ls, nlines, lmap, pl, tw, tid, nt);
}

template <class C, class R>
__device__ void fft2_z_vmul(C* buf, int ldy, int ncol, const R* __restrict__ v, int ldv, const AxisPlan& pz,
                            const C* tw, int tid, int nt) {
    switch (pz.n) {
#define QM_CASE(n)                                                       \
    case n:                                                              \
        if constexpr (Fused<n>::ok) {                                    \
            fft2_z_vmul_ct<C, R, n>(buf, ldy, ncol, v, ldv, tw, tid, nt); \
            return;                                                      \
        }                                                                \
        break;
        QM_FFT_LENGTHS(QM_CASE)
#undef QM_CASE
        default: break;
    }
    fft_z_vmul<C, R>(buf, ldy, ncol, nullptr, ncol, v, ldv, pz, tw, tid, nt);
}

// whether the two-register-pass code serves a runtime length (host side)
inline bool fused_length(int n) {
    switch (n) {
#define QM_CASE(n) \
    case n: return Fused<n>::ok;
        QM_FFT_LENGTHS(QM_CASE)
#undef QM_CASE
        default: return false;
    }
}

// x sticks per CTA of the stick kernels and the CTA's threads: 32 sticks in both precisions,
// 128 threads in FP32 (small CTAs, many per SM: 6-10 % faster than 64 sticks on 256 threads),
// 256 in FP64
template <class R> constexpr int sticks_per_cta() { return 32; }
template <class R> constexpr int stick_threads() { return sizeof(R) == 4 ? 128 : 256; }
constexpr int kThreads = 256;
constexpr size_t kMaxGridY = 65535;  // largest y extent of a launch grid (bands or pairs per launch)
// resident CTAs the register budget is sized for: FP32 4 (stage-per-pass) or 3 (two register
// passes, groups of up to 18 complex values); FP64 2, which the shared memory of an FP64
// plane or stick tile allows at most anyway (fewer would force spills of the 64-bit values)
template <class R, bool FUSED> constexpr int fft_min_ctas() { return sizeof(R) == 8 ? 2 : (FUSED ? 3 : 4); }

// ---------------------------------------------------------------- K1
// FUSED: the two-register-pass transforms (a separate instantiation, so that the stage-per-pass
// lengths keep their lower register count and higher occupancy)
template <class R, bool FUSED>
__global__ void __launch_bounds__(kThreads, fft_min_ctas<R, FUSED>())
k_stick_inverse(const typename Cx<R>::T* __restrict__ psi, int ld_psi, const int* __restrict__ stick_g0,
                const int2* __restrict__ g_code, int nstick, int nstick_pad, const __grid_constant__ AxisPlan px,
                const typename Cx<R>::T* __restrict__ tw_x, int ldx, typename Cx<R>::T* __restrict__ T, int pair_nb) {
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* lines = reinterpret_cast<C*>(smem_raw);
    C* tw = lines + sticks_per_cta<R>() * ldx;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int b = blockIdx.y;
    const int s0 = blockIdx.x * sticks_per_cta<R>();
    const int ns = min(sticks_per_cta<R>(), nstick - s0);
    const int N1 = px.n;
    for (int i = tid; i < N1; i += nt) tw[i] = tw_x[i];
    for (int i = tid; i < ns * ldx; i += nt) lines[i] = mk<C>(0, 0);
    __syncthreads();
    const int gb = __ldg(stick_g0 + s0), ge = __ldg(stick_g0 + s0 + ns);
    if (pair_nb) {
        // Gamma-point real wavefunctions: bands 2b and 2b+1 in one transform, psi_a + i psi_b
        const C* sa = psi + (size_t)(2 * b) * ld_psi;
        const C* sb = 2 * b + 1 < pair_nb ? sa + ld_psi : nullptr;
        for (int g = gb + tid; g < ge; g += nt) {
            int2 c = __ldg(g_code + g);
            const C a = sa[g];
            const C v = sb ? sb[g] : mk<C>(0, 0);
            lines[(c.x - s0) * ldx + c.y] = mk<C>(a.x - v.y, a.y + v.x);
        }
    } else {
        const C* src = psi + (size_t)b * ld_psi;
        for (int g = gb + tid; g < ge; g += nt) {
            int2 c = __ldg(g_code + g);
            lines[(c.x - s0) * ldx + c.y] = src[g];
        }
    }
    __syncthreads();
    if constexpr (FUSED)
        fft2_lines<C, +1, true, false>(lines, 1, ldx, ns, nullptr, px, tw, tid, nt);
    else
        fft_lines<C, +1, true, false>(lines, 1, ldx, ns, nullptr, px, tw, tid, nt);
    C* dst = T + (size_t)b * N1 * nstick_pad + s0;
    for (int i = tid; i < N1 * ns; i += nt) {
        int p = i / ns, l = i - p * ns;
        dst[(size_t)p * nstick_pad + l] = lines[l * ldx + p];
    }
}

// ---------------------------------------------------------------- K2
template <class R, bool FUSED>
__global__ void __launch_bounds__(kThreads, fft_min_ctas<R, FUSED>())
k_plane(typename Cx<R>::T* __restrict__ T, int nstick, int nstick_pad, const int* __restrict__ stick_plane,
        const int* __restrict__ rows, int nrow, const __grid_constant__ AxisPlan py, const __grid_constant__ AxisPlan pz,
        const typename Cx<R>::T* __restrict__ tw_y, const typename Cx<R>::T* __restrict__ tw_z, int ldy,
        const R* __restrict__ Vt, int N1) {
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N2 = py.n, N3 = pz.n;
    C* plane = reinterpret_cast<C*>(smem_raw);
    C* twy = plane + N3 * ldy;
    C* twz = twy + N2;
    int* srow = reinterpret_cast<int*>(twz + N3);  // the active rows (read in every row pass)
    const int tid = threadIdx.x, nt = blockDim.x;
    const int p1 = blockIdx.x, b = blockIdx.y;
    for (int i = tid; i < N2; i += nt) twy[i] = tw_y[i];
    for (int i = tid; i < N3; i += nt) twz[i] = tw_z[i];
    for (int i = tid; i < nrow; i += nt) srow[i] = __ldg(rows + i);
    for (int i = tid; i < N3 * ldy; i += nt) plane[i] = mk<C>(0, 0);
    __syncthreads();
    C* Tp = T + ((size_t)b * N1 + p1) * nstick_pad;
    for (int s = tid; s < nstick; s += nt) plane[__ldg(stick_plane + s)] = Tp[s];
    __syncthreads();
    // inverse y on the active rows; z on every column: inverse, V(r)/N_r (in the permuted,
    // digit-reversed order of all three axes), forward; forward y on the active rows
    if constexpr (FUSED) {
        fft2_lines<C, +1, true, false>(plane, 1, ldy, nrow, srow, py, twy, tid, nt);
        fft2_z_vmul<C, R>(plane, ldy, N2, Vt + (size_t)p1 * N3 * N2, N2, pz, twz, tid, nt);
        fft2_lines<C, -1, false, false>(plane, 1, ldy, nrow, srow, py, twy, tid, nt);
    } else {
        fft_lines<C, +1, true, false>(plane, 1, ldy, nrow, srow, py, twy, tid, nt);
        fft_z_vmul<C, R>(plane, ldy, N2, nullptr, N2, Vt + (size_t)p1 * N3 * N2, N2, pz, twz, tid, nt);
        fft_lines<C, -1, false, false>(plane, 1, ldy, nrow, srow, py, twy, tid, nt);
    }
    for (int s = tid; s < nstick; s += nt) Tp[s] = plane[__ldg(stick_plane + s)];
}

// ---------------------------------------------------------------- K3
template <class R, bool FUSED>
__global__ void __launch_bounds__(kThreads, fft_min_ctas<R, FUSED>())
k_stick_forward(const typename Cx<R>::T* __restrict__ T, int nstick, int nstick_pad,
                const int* __restrict__ stick_g0, const int2* __restrict__ g_code, const R* __restrict__ kin,
                const __grid_constant__ AxisPlan px, const typename Cx<R>::T* __restrict__ tw_x, int ldx,
                const typename Cx<R>::T* __restrict__ psi, int ld_psi, typename Cx<R>::T* __restrict__ out,
                int ld_out, int accumulate) {
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* lines = reinterpret_cast<C*>(smem_raw);
    C* tw = lines + sticks_per_cta<R>() * ldx;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int b = blockIdx.y;
    const int s0 = blockIdx.x * sticks_per_cta<R>();
    const int ns = min(sticks_per_cta<R>(), nstick - s0);
    const int N1 = px.n;
    for (int i = tid; i < N1; i += nt) tw[i] = tw_x[i];
    const C* srcT = T + (size_t)b * N1 * nstick_pad + s0;
    for (int i = tid; i < N1 * ns; i += nt) {
        int p = i / ns, l = i - p * ns;
        lines[l * ldx + p] = srcT[(size_t)p * nstick_pad + l];
    }
    __syncthreads();
    if constexpr (FUSED)
        fft2_lines<C, -1, false, false>(lines, 1, ldx, ns, nullptr, px, tw, tid, nt);
    else
        fft_lines<C, -1, false, false>(lines, 1, ldx, ns, nullptr, px, tw, tid, nt);
    const int gb = __ldg(stick_g0 + s0), ge = __ldg(stick_g0 + s0 + ns);
    const C* ps = psi + (size_t)b * ld_psi;
    C* po = out + (size_t)b * ld_out;
    for (int g = gb + tid; g < ge; g += nt) {
        int2 c = __ldg(g_code + g);
        C x = lines[(c.x - s0) * ldx + c.y];
        C y = ps[g];
        R k = __ldg(kin + g);
        C r = mk<C>(x.x + k * y.x, x.y + k * y.y);
        if (accumulate) r = add(r, po[g]);
        po[g] = r;
    }
}

// ---------------------------------------------------------------- K3, Gamma-point real wavefunctions
// One CTA per (tile of kGammaTile sticks, band pair b): the tile holds every stick together with
// the stick of the opposite (i2, i3), so F(G) and F(-G) of the pair's transform F = V(psi_a +
// i psi_b) are both in shared memory after the x-forward pass.  For real-space-real psi_a, psi_b
// (psi(-G) = conj psi(G)) the two products separate as
//     (V psi_a)(G) = (F(G) + conj F(-G)) / 2,   (V psi_b)(G) = (F(G) - conj F(-G)) / (2i),
// then the kinetic term is added (and the nonlocal part already in `out` when accumulate).
template <class R, bool FUSED>
__global__ void __launch_bounds__(kThreads, fft_min_ctas<R, FUSED>())
k_stick_forward_gamma(const typename Cx<R>::T* __restrict__ T, int nstick_pad, const int2* __restrict__ gtile,
                      const int* __restrict__ stick_g0, const int2* __restrict__ g_code, const R* __restrict__ kin,
                      const __grid_constant__ AxisPlan px, const typename Cx<R>::T* __restrict__ tw_x, int ldx,
                      const typename Cx<R>::T* __restrict__ psi, int ld_psi, typename Cx<R>::T* __restrict__ out,
                      int ld_out, int accumulate, int nb) {
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* lines = reinterpret_cast<C*>(smem_raw);
    C* tw = lines + kGammaTile * ldx;
    __shared__ int2 slot[kGammaTile];
    __shared__ int gstart[kGammaTile], goff[kGammaTile + 1];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int b = blockIdx.y;
    const int N1 = px.n;
    for (int i = tid; i < N1; i += nt) tw[i] = tw_x[i];
    if (tid < kGammaTile) {
        const int2 sl = __ldg(gtile + (size_t)blockIdx.x * kGammaTile + tid);
        slot[tid] = sl;
        const int g0 = sl.x >= 0 ? __ldg(stick_g0 + sl.x) : 0;
        gstart[tid] = g0;
        goff[tid + 1] = sl.x >= 0 ? __ldg(stick_g0 + sl.x + 1) - g0 : 0;
    }
    __syncthreads();
    if (tid == 0) {
        goff[0] = 0;
        for (int l = 0; l < kGammaTile; ++l) goff[l + 1] += goff[l];
    }
    const C* srcT = T + (size_t)b * N1 * nstick_pad;
    for (int i = tid; i < N1 * kGammaTile; i += nt) {
        const int p = i / kGammaTile, l = i - p * kGammaTile;
        const int st = slot[l].x;
        lines[l * ldx + p] = st >= 0 ? srcT[(size_t)p * nstick_pad + st] : mk<C>(0, 0);
    }
    __syncthreads();
    if constexpr (FUSED)
        fft2_lines<C, -1, false, false>(lines, 1, ldx, kGammaTile, nullptr, px, tw, tid, nt);
    else
        fft_lines<C, -1, false, false>(lines, 1, ldx, kGammaTile, nullptr, px, tw, tid, nt);
    const int ba = 2 * b;
    const bool has_b = ba + 1 < nb;
    const C* pa = psi + (size_t)ba * ld_psi;
    C* oa = out + (size_t)ba * ld_out;
    const int total = goff[kGammaTile];
    for (int t = tid; t < total; t += nt) {
        int lo = 0, hi = kGammaTile;  // slot l with goff[l] <= t < goff[l + 1]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (goff[mid] <= t) lo = mid;
            else hi = mid;
        }
        const int l = lo;
        const int g = gstart[l] + (t - goff[l]);
        const int x = __ldg(g_code + g).y;
        const int xm = x ? N1 - x : 0;
        const C F = lines[l * ldx + x];
        const C Fm = lines[slot[l].y * ldx + xm];
        const R k = __ldg(kin + g);
        const R h = (R)0.5;
        C y = pa[g];
        C r = mk<C>(h * (F.x + Fm.x) + k * y.x, h * (F.y - Fm.y) + k * y.y);
        if (accumulate) r = add(r, oa[g]);
        oa[g] = r;
        if (has_b) {
            y = pa[(size_t)ld_psi + g];
            r = mk<C>(h * (F.y + Fm.y) + k * y.x, h * (Fm.x - F.x) + k * y.y);
            if (accumulate) r = add(r, oa[(size_t)ld_out + g]);
            oa[(size_t)ld_out + g] = r;
        }
    }
}

// ---------------------------------------------------------------- V layout
template <class R>
__global__ void k_vt(const double* __restrict__ V, R* __restrict__ Vt, int N1, int N2, int N3,
                     const int* __restrict__ rev1, const int* __restrict__ rev2, const int* __restrict__ rev3,
                     double scale) {
    const size_t nr = (size_t)N1 * N2 * N3;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nr; i += (size_t)gridDim.x * blockDim.x) {
        int p2 = (int)(i % N2);
        size_t q = i / N2;
        int p3 = (int)(q % N3);
        int p1 = (int)(q / N3);
        size_t src = (size_t)__ldg(rev1 + p1) + (size_t)N1 * ((size_t)__ldg(rev2 + p2) + (size_t)N2 * __ldg(rev3 + p3));
        Vt[i] = (R)(__ldg(V + src) * scale);
    }
}

// Threads of a k_plane CTA: 192 where that keeps at least 90 % of the resident threads of
// 256-thread CTAs (more, smaller CTAs per SM: each barrier of a pass waits for fewer warps;
// measured 4-6 % faster on the 72^3 and 96x96x48 grids), else 256 (e.g. the 90^3 plane, whose
// shared memory allows only three CTAs per SM).  The transforms do not depend on the choice.
inline int plane_threads(const void* kernel, size_t smem) {
    int o256 = 0, o192 = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o256, kernel, 256, smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o192, kernel, 192, smem) != cudaSuccess) {
        cudaGetLastError();
        return kThreads;
    }
    return 192 * o192 * 10 >= 256 * o256 * 9 ? 192 : 256;
}

// ---------------------------------------------------------------- per-precision launch sequences
// wait_k3: event the stream waits for before the first x-forward pass (the nonlocal part
// running concurrently on another stream); accumulate: the x-forward pass adds to `out`.
// gamma: the Gamma-point real-wavefunction form (two bands per transform, k_stick_forward_gamma)
template <class R>
qm_status local_kinetic_impl(qm_gspace g, int ik, int nb, const void* psi, int ld_psi, const void* vt,
                                    void* out, int ld_out, void* tbuf, size_t tbuf_bytes, cudaStream_t s,
                                    cudaEvent_t wait_k3, bool accumulate, bool gamma) {
    using C = typename Cx<R>::T;
    const KTables& kt = g->k[ik];
    const int N1 = g->n[0], N2 = g->n[1], N3 = g->n[2];
    const size_t per_band = (size_t)N1 * kt.nstick_pad * sizeof(C);
    if (gamma && !kt.gamma) return fail(QM_ERR_ARG, "FFT path: the k-point is not the Gamma point");
    const int ntr = gamma ? (nb + 1) / 2 : nb;  // transforms (band pairs in the Gamma form)
    // transforms per launch: the stick buffer's budget, at most the 65535 CTAs a grid's y extent allows
    const int nbc = (int)std::max<size_t>(1, std::min<size_t>(std::min<size_t>((size_t)ntr, tbuf_bytes / per_band),
                                                              kMaxGridY));
    const size_t sm_stick = (size_t)(sticks_per_cta<R>() * g->ldx + N1) * sizeof(C);
    const size_t sm_plane = (size_t)(N3 * g->ldy + N2 + N3) * sizeof(C) + (size_t)N3 * sizeof(int);
    qm_status st;
    const bool fx = fused_length(N1), fyz = fused_length(N2) || fused_length(N3);
    auto kin_ = fx ? k_stick_inverse<R, true> : k_stick_inverse<R, false>;
    auto kfw_ = fx ? k_stick_forward<R, true> : k_stick_forward<R, false>;
    auto kfg_ = fx ? k_stick_forward_gamma<R, true> : k_stick_forward_gamma<R, false>;
    auto kpl_ = fyz ? k_plane<R, true> : k_plane<R, false>;
    static_assert(kGammaTile == sticks_per_cta<R>(), "the Gamma tiles use the stick kernels' shared memory");
    if ((st = allow_dynamic_smem((const void*)kpl_, sm_plane, "qm_hpsi: FFT plane in shared memory")) ||
        (st = allow_dynamic_smem((const void*)kin_, sm_stick, "qm_hpsi: FFT sticks in shared memory")) ||
        (st = allow_dynamic_smem(gamma ? (const void*)kfg_ : (const void*)kfw_, sm_stick,
                                 "qm_hpsi: FFT sticks in shared memory")))
        return st;
    const int nt_plane = plane_threads((const void*)kpl_, sm_plane);
    const int ntile = (kt.nstick + sticks_per_cta<R>() - 1) / sticks_per_cta<R>();
    const C* tw_x = (const C*)(sizeof(R) == 8 ? (const void*)g->tw64[0] : (const void*)g->tw32[0]);
    const C* tw_y = (const C*)(sizeof(R) == 8 ? (const void*)g->tw64[1] : (const void*)g->tw32[1]);
    const C* tw_z = (const C*)(sizeof(R) == 8 ? (const void*)g->tw64[2] : (const void*)g->tw32[2]);
    const R* kin = (const R*)(sizeof(R) == 8 ? (const void*)kt.kin : (const void*)kt.kin_f);
    C* T = (C*)tbuf;
    for (int b0 = 0; b0 < ntr; b0 += nbc) {
        const int nbx = std::min(nbc, ntr - b0);
        const int band0 = gamma ? 2 * b0 : b0;
        const int nbands = gamma ? std::min(2 * nbx, nb - band0) : nbx;
        const C* ps = (const C*)psi + (size_t)band0 * ld_psi;
        C* po = (C*)out + (size_t)band0 * ld_out;
        {
            ProfScope pf(PF_STICK_INV, s);
            kin_<<<dim3(ntile, nbx), stick_threads<R>(), sm_stick, s>>>(
                ps, ld_psi, kt.stick_g0, kt.g_code, kt.nstick, kt.nstick_pad, g->plan[0], tw_x, g->ldx, T,
                gamma ? nbands : 0);
        }
        {
            ProfScope pf(PF_PLANE, s);
            kpl_<<<dim3(N1, nbx), nt_plane, sm_plane, s>>>(
                T, kt.nstick, kt.nstick_pad, kt.stick_plane, kt.rows, kt.nrow, g->plan[1], g->plan[2], tw_y, tw_z,
                g->ldy, (const R*)vt, N1);
        }
        if (wait_k3 && b0 == 0) {
            cudaError_t e = cudaStreamWaitEvent(s, wait_k3, 0);
            if (e != cudaSuccess) return cuda_check(e, "FFT path: wait for the nonlocal part");
        }
        {
            ProfScope pf(PF_STICK_FWD, s);
            if (gamma)
                kfg_<<<dim3(kt.ngtile, nbx), stick_threads<R>(), sm_stick, s>>>(
                    T, kt.nstick_pad, kt.gtile, kt.stick_g0, kt.g_code, kin, g->plan[0], tw_x, g->ldx, ps, ld_psi, po,
                    ld_out, accumulate ? 1 : 0, nbands);
            else
                kfw_<<<dim3(ntile, nbx), stick_threads<R>(), sm_stick, s>>>(
                    T, kt.nstick, kt.nstick_pad, kt.stick_g0, kt.g_code, kin, g->plan[0], tw_x, g->ldx, ps, ld_psi,
                    po, ld_out, accumulate ? 1 : 0);
        }
    }
    return cuda_check(cudaGetLastError(), "FFT path launch");
}

template <class R>
qm_status local_kinetic_tab_impl(const DevTables& t, int nb, const void* psi, int ld_psi, const void* vt,
                                        void* out, int ld_out, void* tbuf, size_t tbuf_bytes, cudaStream_t s) {
    using C = typename Cx<R>::T;
    const int N1 = t.n[0], N2 = t.n[1], N3 = t.n[2];
    const size_t per_band = (size_t)N1 * t.nstick_pad * sizeof(C);
    if (tbuf_bytes < per_band) return fail(QM_ERR_ARG, "stick buffer smaller than one band");
    const int nbc = (int)std::max<size_t>(1, std::min<size_t>(std::min<size_t>((size_t)nb, tbuf_bytes / per_band),
                                                              kMaxGridY));
    const size_t sm_stick = (size_t)(sticks_per_cta<R>() * t.ldx + N1) * sizeof(C);
    const size_t sm_plane = (size_t)(N3 * t.ldy + N2 + N3) * sizeof(C) + (size_t)N3 * sizeof(int);
    qm_status st;
    const bool fx = fused_length(N1), fyz = fused_length(N2) || fused_length(N3);
    auto kin_ = fx ? k_stick_inverse<R, true> : k_stick_inverse<R, false>;
    auto kfw_ = fx ? k_stick_forward<R, true> : k_stick_forward<R, false>;
    auto kpl_ = fyz ? k_plane<R, true> : k_plane<R, false>;
    if ((st = allow_dynamic_smem((const void*)kpl_, sm_plane, "FFT plane in shared memory")) ||
        (st = allow_dynamic_smem((const void*)kin_, sm_stick, "FFT sticks in shared memory")) ||
        (st = allow_dynamic_smem((const void*)kfw_, sm_stick, "FFT sticks in shared memory")))
        return st;
    const int nt_plane = plane_threads((const void*)kpl_, sm_plane);
    const int ntile = (t.nstick + sticks_per_cta<R>() - 1) / sticks_per_cta<R>();
    const C* tw_x = (const C*)t.tw[0];
    const C* tw_y = (const C*)t.tw[1];
    const C* tw_z = (const C*)t.tw[2];
    const R* kin = (const R*)t.kin;
    C* T = (C*)tbuf;
    for (int b0 = 0; b0 < nb; b0 += nbc) {
        const int nbx = std::min(nbc, nb - b0);
        const C* ps = (const C*)psi + (size_t)b0 * ld_psi;
        C* po = (C*)out + (size_t)b0 * ld_out;
        {
            ProfScope pf(PF_STICK_INV, s);
            kin_<<<dim3(ntile, nbx), stick_threads<R>(), sm_stick, s>>>(
                ps, ld_psi, t.stick_g0, t.g_code, t.nstick, t.nstick_pad, t.plan[0], tw_x, t.ldx, T, 0);
        }
        {
            ProfScope pf(PF_PLANE, s);
            kpl_<<<dim3(N1, nbx), nt_plane, sm_plane, s>>>(
                T, t.nstick, t.nstick_pad, t.stick_plane, t.rows, t.nrow, t.plan[1], t.plan[2], tw_y, tw_z, t.ldy,
                (const R*)vt, N1);
        }
        {
            ProfScope pf(PF_STICK_FWD, s);
            kfw_<<<dim3(ntile, nbx), stick_threads<R>(), sm_stick, s>>>(
                T, t.nstick, t.nstick_pad, t.stick_g0, t.g_code, kin, t.plan[0], tw_x, t.ldx, ps, ld_psi, po, ld_out, 0);
        }
    }
    return cuda_check(cudaGetLastError(), "FFT path launch");
}

}  // namespace qm
