// qm_hpsi_noalloc: the H psi of qm_hpsi for callers that must not allocate device memory.
//
// Who needs it: code that runs under an allocator owning the whole device heap (a host
// framework that reserves the free memory up front and forbids cudaMalloc afterwards),
// and latency-critical loops in which a cudaMalloc/cudaFree would synchronise the device
// or fail for lack of free memory.  Such callers still own and pass every input and
// output; the scratch this call needs (the gspace tables of the k-point, V(r) in the FFT
// layout, the projections and split-K partials, the stick buffer) lives in one fixed,
// file-scope device array below, reserved when the library is loaded on a GPU and held
// until the process exits.
//
// Rules of use:
//  - every call resolves the array's device address (cudaGetSymbolAddress, no allocation);
//    the first call on a device may load the library's device code there, so make that first
//    call outside any stream capture;
//  - every call, from any handle or thread, shares the one array: calls whose work
//    overlaps on the GPU (different streams, or different threads without ordering)
//    race on it; order them on one stream;
//  - nothing in the array has to start at zero: each call writes every scratch byte it
//    reads (tables are copied in, the stick buffer and partial sums are fully written);
//  - the k-point's FFT tables: if the handle already holds them on the device (an earlier
//    qm_hpsi or qm_davidson call with the handle uploaded them), they are read in place and the
//    call only queues work on the stream; otherwise they are copied on every call from the
//    handle's host copies into the scratch array (pageable host memory, so the host waits
//    until the stream's earlier work is done before each copy);
//  - QM_MIXED: the FFT path is the FP32 one of qm_hpsi; the nonlocal projection and
//    application are FP32 SIMT products (not the tensor-core BF16x3 split of qm_hpsi, whose
//    operand planes would need scratch of their own);
//  - problems whose scratch exceeds QM_HPSI_NOALLOC_SCRATCH_BYTES are rejected with
//    QM_ERR_ARG and a message giving the bytes needed.
// No cudaMalloc, cudaFree or other allocating routine is called on this path.
#include <algorithm>
#include <cstring>

#include "qm_internal.h"

namespace qm {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[QM_HPSI_NOALLOC_SCRATCH_BYTES];

// device address of the scratch array on the current device, resolved on every call (a
// cached address could outlive a module reload after the context is torn down)
qm_status scratch_address(void** out) {
    void* p = nullptr;
    qm_status st = cuda_check(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress(noalloc scratch)");
    if (st) return st;
    *out = p;
    return QM_OK;
}

__global__ void k_to_float(const double* __restrict__ in, float* __restrict__ out, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = (float)in[i];
}

struct Carve {
    size_t off = 0;
    size_t take(size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    }
};

}  // namespace
}  // namespace qm

using namespace qm;

extern "C" qm_status qm_hpsi_noalloc(qm_gspace g, int ik, int nb, const void* psi, int ld_psi,
                                     const double* vloc_r, int nproj, const void* beta, int ld_beta,
                                     const double* D, void* out, int ld_out, qm_precision prec, void* stream) {
    clear_error();
    if (!g) return fail(QM_ERR_ARG, "qm_hpsi_noalloc: NULL gspace");
    if (ik < 0 || ik >= g->nk) return fail(QM_ERR_ARG, "qm_hpsi_noalloc: ik out of range");
    if (nb < 0 || nproj < 0) return fail(QM_ERR_ARG, "qm_hpsi_noalloc: negative nb or nproj");
    if (prec != QM_FP64 && prec != QM_MIXED) return fail(QM_ERR_ARG, "qm_hpsi_noalloc: unknown precision");
    if (nb == 0) return QM_OK;
    const KTables& kt = g->k[ik];
    const int npw = kt.npw;
    if (!psi || !out || !vloc_r) return fail(QM_ERR_ARG, "qm_hpsi_noalloc: NULL psi, out or vloc_r");
    if (ld_psi < npw || ld_out < npw) return fail(QM_ERR_ARG, "qm_hpsi_noalloc: leading dimension < npw");
    if (nproj > 0 && (!beta || !D)) return fail(QM_ERR_ARG, "qm_hpsi_noalloc: NULL beta or D with nproj > 0");
    if (nproj > 0 && ld_beta < npw) return fail(QM_ERR_ARG, "qm_hpsi_noalloc: ld_beta < npw");
    const bool fp32 = prec == QM_MIXED;
    const size_t cs = fp32 ? sizeof(float2) : sizeof(double2);
    const size_t rs = fp32 ? sizeof(float) : sizeof(double);
    if (((uintptr_t)psi | (uintptr_t)out | (nproj > 0 ? (uintptr_t)beta : 0)) % cs)
        return fail(QM_ERR_ARG, "qm_hpsi_noalloc: psi/out/beta not aligned to the complex element size");
    {
        const char* a0 = (const char*)psi;
        const char* a1 = a0 + ((size_t)(nb - 1) * ld_psi + npw) * cs;
        const char* b0 = (const char*)out;
        const char* b1 = b0 + ((size_t)(nb - 1) * ld_out + npw) * cs;
        if (a0 < b1 && b0 < a1) return fail(QM_ERR_ARG, "qm_hpsi_noalloc: out overlaps psi");
    }
    const int N1 = g->n[0], N2 = g->n[1], N3 = g->n[2];
    const size_t nr = (size_t)N1 * N2 * N3;
    const size_t per_band = (size_t)N1 * kt.nstick_pad * cs;

    // the handle's device tables, when an earlier call uploaded them to this device
    int cur_dev = -1;
    if (cudaGetDevice(&cur_dev) != cudaSuccess) return fail(QM_ERR_CUDA, "qm_hpsi_noalloc: cudaGetDevice");
    const bool in_place = g->uploaded && g->device == cur_dev;
    // scratch layout: tables (unless in place) | Vt | P | stick buffer (>= 1 band) | split-K partials (what is left)
    Carve c;
    const bool copy = !in_place;
    const size_t o_g0 = c.take(copy ? sizeof(int) * kt.h_g0.size() : 0);
    const size_t o_plane = c.take(copy ? sizeof(int) * kt.h_plane.size() : 0);
    const size_t o_rows = c.take(copy ? sizeof(int) * kt.h_rows.size() : 0);
    const size_t o_code = c.take(copy ? sizeof(int2) * kt.h_code.size() : 0);
    const size_t o_kin64 = c.take(copy ? sizeof(double) * npw : 0);
    const size_t o_kin32 = c.take(copy && fp32 ? sizeof(float) * npw : 0);
    size_t o_tw64[3], o_tw32[3], o_rev[3];
    for (int d = 0; d < 3; ++d) {
        o_tw64[d] = c.take(copy ? sizeof(double2) * g->n[d] : 0);
        o_tw32[d] = c.take(copy && fp32 ? sizeof(float2) * g->n[d] : 0);
        o_rev[d] = c.take(copy ? sizeof(int) * g->n[d] : 0);
    }
    const size_t o_vt = c.take(nr * rs);
    const size_t o_p = c.take((size_t)nproj * nb * cs);
    const size_t need_min = c.off + per_band;
    if (need_min > (size_t)QM_HPSI_NOALLOC_SCRATCH_BYTES) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "qm_hpsi_noalloc: this problem needs at least %zu bytes of scratch; the fixed scratch holds %zu "
                 "(QM_HPSI_NOALLOC_SCRATCH_BYTES): use qm_hpsi",
                 need_min, (size_t)QM_HPSI_NOALLOC_SCRATCH_BYTES);
        return fail(QM_ERR_ARG, msg);
    }
    const size_t room = (size_t)QM_HPSI_NOALLOC_SCRATCH_BYTES - c.off;
    // stick buffer: up to the L2-sized chunk of qm_hpsi, leaving room for the partial sums
    const size_t pbytes_split = (size_t)nproj * nb * cs;
    size_t t_bytes = std::min(room, std::max(per_band, std::min<size_t>(48ull << 20, (size_t)nb * per_band)));
    t_bytes = t_bytes / per_band * per_band;
    const size_t o_t = c.take(t_bytes);
    int splits = 1;
    size_t o_part = 0;
    if (nproj > 0 && c.off < (size_t)QM_HPSI_NOALLOC_SCRATCH_BYTES) {
        const size_t left = (size_t)QM_HPSI_NOALLOC_SCRATCH_BYTES - c.off;
        splits = (int)std::min<size_t>((size_t)zgemm_cn_splits(nproj, nb, npw), left / std::max<size_t>(1, pbytes_split));
        splits = std::max(1, splits);
        if (splits > 1) o_part = c.take((size_t)splits * pbytes_split);
    }

    void* base_v = nullptr;
    qm_status st = scratch_address(&base_v);
    if (st) return st;
    char* base = (char*)base_v;
    cudaStream_t s = (cudaStream_t)stream;
    auto up = [&](size_t off, const void* src, size_t bytes) -> qm_status {
        if (bytes == 0) return QM_OK;
        return cuda_check(cudaMemcpyAsync(base + off, src, bytes, cudaMemcpyHostToDevice, s), "noalloc table copy");
    };
    DevTables t;
    if (in_place) {
        for (int d = 0; d < 3; ++d) {
            t.tw[d] = fp32 ? (const void*)g->tw32[d] : (const void*)g->tw64[d];
            t.rev[d] = g->rev[d];
        }
        t.stick_g0 = kt.stick_g0;
        t.stick_plane = kt.stick_plane;
        t.rows = kt.rows;
        t.g_code = kt.g_code;
        t.kin = fp32 ? (const void*)kt.kin_f : (const void*)kt.kin;
    } else if ((st = up(o_g0, kt.h_g0.data(), sizeof(int) * kt.h_g0.size())) ||
        (st = up(o_plane, kt.h_plane.data(), sizeof(int) * kt.h_plane.size())) ||
        (st = up(o_rows, kt.h_rows.data(), sizeof(int) * kt.h_rows.size())) ||
        (st = up(o_code, kt.h_code.data(), sizeof(int2) * kt.h_code.size())) ||
        (st = up(o_kin64, kt.h_kin.data(), sizeof(double) * npw))) {
        return st;
    }
    if (copy) {
        for (int d = 0; d < 3; ++d)
            if ((st = up(o_tw64[d], g->h_tw[d].data(), sizeof(double2) * g->n[d])) ||
                (st = up(o_rev[d], g->h_rev[d].data(), sizeof(int) * g->n[d])))
                return st;
        if (fp32) {
            k_to_float<<<(npw + 255) / 256, 256, 0, s>>>((const double*)(base + o_kin64), (float*)(base + o_kin32), npw);
            count_launch(1);
            for (int d = 0; d < 3; ++d) {
                k_to_float<<<1, 256, 0, s>>>((const double*)(base + o_tw64[d]), (float*)(base + o_tw32[d]), 2 * g->n[d]);
                count_launch(1);
            }
        }
        for (int d = 0; d < 3; ++d) {
            t.tw[d] = base + (fp32 ? o_tw32[d] : o_tw64[d]);
            t.rev[d] = (const int*)(base + o_rev[d]);
        }
        t.stick_g0 = (const int*)(base + o_g0);
        t.stick_plane = (const int*)(base + o_plane);
        t.rows = (const int*)(base + o_rows);
        t.g_code = (const int2*)(base + o_code);
        t.kin = base + (fp32 ? o_kin32 : o_kin64);
    }
    for (int d = 0; d < 3; ++d) {
        t.n[d] = g->n[d];
        t.plan[d] = g->plan[d];
    }
    t.ldx = g->ldx;
    t.ldy = g->ldy;
    t.nstick = kt.nstick;
    t.nstick_pad = kt.nstick_pad;
    t.nrow = kt.nrow;

    void* vt = base + o_vt;
    void* P = base + o_p;
    void* T = base + o_t;
    void* part = splits > 1 ? base + o_part : nullptr;
    if ((st = launch_vt_prepare_tab(t, vloc_r, vt, fp32, s))) return st;
    if (nproj > 0) {
        if (fp32)
            st = cgemm_cn(nproj, nb, npw, (const float2*)beta, ld_beta, (const float2*)psi, ld_psi, (float2*)P, nb,
                          (float2*)part, splits, s);
        else
            st = zgemm_cn(nproj, nb, npw, (const double2*)beta, ld_beta, (const double2*)psi, ld_psi, (double2*)P,
                          nb, (double2*)part, splits, s);
        if (st) return st;
    }
    if ((st = launch_local_kinetic_tab(t, nb, psi, ld_psi, vt, out, ld_out, T, t_bytes, fp32, s))) return st;
    if (nproj > 0) {
        if (fp32)
            st = cgemm_tn(nb, npw, nproj, (const float2*)P, nb, D, (const float2*)beta, ld_beta, (float2*)out,
                          ld_out, true, s);
        else
            st = zgemm_tn(nb, npw, nproj, (const double2*)P, nb, D, (const double2*)beta, ld_beta, (double2*)out,
                          ld_out, true, s);
        if (st) return st;
    }
    return cuda_check(cudaGetLastError(), "qm_hpsi_noalloc launches");
}
