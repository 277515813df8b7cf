// Host-side G-space construction: FFT grid, plane-wave sphere per k-point, x-stick
// tables and mixed-radix FFT plans, uploaded to the device once per handle.
//
// Follows the truncation of Sec. 2.2 (|k+G|^2/2 <= E_cut, potential up to 4 E_cut) and
// the GSpace of Sec. 4.3.2 (plane waves listed with G_1 fastest); the stick pruning of
// Sec. 4.3.3 (1D FFTs only on sticks that hold a plane wave) with sticks along x as in
// the paper's Fig. 1.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>

#include <new>

#include "qm_internal.h"

namespace qm {

static thread_local std::string g_last_error;

qm_status fail(qm_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}
void clear_error() { g_last_error.clear(); }

qm_status cuda_check(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return QM_OK;
    cudaGetLastError();  // clear a sticky launch error where possible
    return fail(e == cudaErrorMemoryAllocation ? QM_ERR_OOM : QM_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

// Grow-only workspace.  Its first kWsHeader bytes are a header that survives regrowth (the
// handle's sticky device error word lives there, see qm_hpsi_check); a new workspace starts
// with a zero header.
static qm_status grow(Workspace& ws, size_t bytes, cudaStream_t stream) {
    bytes = std::max(bytes, kWsHeader);
    if (ws.bytes >= bytes) return QM_OK;
    size_t want = align_up(bytes + bytes / 8, 1 << 20);
    void* fresh = nullptr;
    qm_status st;
    if (ws.ptr && (st = cuda_check(cudaStreamSynchronize(stream), "workspace sync"))) return st;
    if ((st = cuda_check(cudaMalloc(&fresh, want), "workspace cudaMalloc"))) return st;
    st = ws.ptr ? cuda_check(cudaMemcpy(fresh, ws.ptr, kWsHeader, cudaMemcpyDeviceToDevice), "workspace header")
                : cuda_check(cudaMemset(fresh, 0, kWsHeader), "workspace header");
    if (st) {
        cudaFree(fresh);
        return st;
    }
    if (ws.ptr) cudaFree(ws.ptr);
    ws.ptr = fresh;
    ws.bytes = want;
    return QM_OK;
}

qm_status allow_dynamic_smem(const void* kernel, size_t need, const char* what) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> done;  // (kernel, device) -> limit set
    int dev = 0;
    qm_status st = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    if (st) return st;
    int max_dyn = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = done.find({kernel, dev});
        if (it != done.end()) {
            max_dyn = it->second;
        } else {
            int optin = 0;
            cudaFuncAttributes fa{};
            if ((st = cuda_check(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), what)) ||
                (st = cuda_check(cudaFuncGetAttributes(&fa, kernel), what)))
                return st;
            max_dyn = optin - (int)fa.sharedSizeBytes;
            if ((st = cuda_check(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn),
                                 what)))
                return st;
            done[{kernel, dev}] = max_dyn;
        }
    }
    if ((long long)need > (long long)max_dyn)
        return fail(QM_ERR_UNSUPPORTED, std::string(what) + ": needs more shared memory than a CTA can have");
    return QM_OK;
}

int device_sms() {
    static std::mutex mu;
    static std::map<int, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    cache[dev] = n;
    return n;
}

qm_status ensure_workspace(qm_gspace g, size_t bytes, cudaStream_t stream) { return grow(g->ws, bytes, stream); }
qm_status ensure_dav_workspace(qm_gspace g, size_t bytes, cudaStream_t stream) { return grow(g->dws, bytes, stream); }

static bool smooth235(int n) {
    if (n <= 0) return false;
    for (int p : {2, 3, 5})
        while (n % p == 0) n /= p;
    return n == 1;
}

static void inv3_transpose_2pi(const double a[9], double b[9]) {
    // b rows = 2 pi (A^-1)^T rows, i.e. b_i . a_j = 2 pi delta_ij
    double c[9];
    c[0] = a[4] * a[8] - a[5] * a[7];
    c[1] = a[5] * a[6] - a[3] * a[8];
    c[2] = a[3] * a[7] - a[4] * a[6];
    c[3] = a[2] * a[7] - a[1] * a[8];
    c[4] = a[0] * a[8] - a[2] * a[6];
    c[5] = a[1] * a[6] - a[0] * a[7];
    c[6] = a[1] * a[5] - a[2] * a[4];
    c[7] = a[2] * a[3] - a[0] * a[5];
    c[8] = a[0] * a[4] - a[1] * a[3];
    double det = a[0] * c[0] + a[1] * c[1] + a[2] * c[2];
    // (A^-1)^T = cofactor matrix / det; row i of the cofactor matrix is c[3i..3i+2]
    const double twopi = 2.0 * M_PI;
    for (int i = 0; i < 9; ++i) b[i] = twopi * c[i] / det;
}

void fft_plan(int n, int order, AxisPlan& p, std::vector<int>& rev) {
    p.n = n;
    p.nst = 0;
    int m = n;
    // radix order 0: 8s, at most one 4 and one 2, 9s, at most one 3, 5s; order 1: the same
    // radices reversed (must match the compile-time plans of the FFT kernels, make_cplan)
    std::vector<int> rs;
    while (m % 8 == 0) { rs.push_back(8); m /= 8; }
    if (m % 4 == 0) { rs.push_back(4); m /= 4; }
    if (m % 2 == 0) { rs.push_back(2); m /= 2; }
    while (m % 9 == 0) { rs.push_back(9); m /= 9; }
    if (m % 3 == 0) { rs.push_back(3); m /= 3; }
    while (m % 5 == 0) { rs.push_back(5); m /= 5; }
    if (order) std::reverse(rs.begin(), rs.end());
    int L = n;
    for (int r : rs) {
        p.r[p.nst] = r;
        p.L[p.nst] = L;
        ++p.nst;
        L /= r;
    }
    // position of natural index k after the in-place DIF stages:
    // pos(k) = M * (k mod r) + pos_sub(k div r), applied recursively over the stages.
    std::vector<int> pos(n);
    for (int k = 0; k < n; ++k) {
        int kk = k, off = 0;
        for (int s = 0; s < p.nst; ++s) {
            int r = p.r[s], Ls = p.L[s], M = Ls / r;
            off += M * (kk % r);
            kk /= r;
        }
        pos[k] = off;
    }
    rev.assign(n, 0);
    for (int k = 0; k < n; ++k) rev[pos[k]] = k;
}

struct PW {
    int64_t idx;
    int m[3];
    double q[3];
    double kin;
};

qm_status ensure_device(qm_gspace g) {
    int dev = 0;
    qm_status st = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    if (st) return st;
    if (g->uploaded) {
        if (dev != g->device) return fail(QM_ERR_ARG, "gspace tables live on another device than the current one");
        return QM_OK;
    }
    auto upload = [&](void** dptr, const void* src, size_t bytes) -> qm_status {
        if (bytes == 0) bytes = 16;
        qm_status s2 = cuda_check(cudaMalloc(dptr, bytes), "gspace table cudaMalloc");
        if (s2) return s2;
        return cuda_check(cudaMemcpy(*dptr, src, bytes, cudaMemcpyHostToDevice), "gspace table upload");
    };
    g->device = dev;
    g->uploaded = true;  // destroy frees whatever was allocated even on partial failure
    for (int d = 0; d < 3; ++d) {
        std::vector<float2> t32(g->n[d]);
        for (int t = 0; t < g->n[d]; ++t) t32[t] = make_float2((float)g->h_tw[d][t].x, (float)g->h_tw[d][t].y);
        if ((st = upload((void**)&g->tw64[d], g->h_tw[d].data(), sizeof(double2) * g->n[d])) ||
            (st = upload((void**)&g->tw32[d], t32.data(), sizeof(float2) * g->n[d])) ||
            (st = upload((void**)&g->rev[d], g->h_rev[d].data(), sizeof(int) * g->n[d])))
            return st;
    }
    for (auto& kt : g->k) {
        std::vector<float> kinf(kt.h_kin.begin(), kt.h_kin.end());
        if ((st = upload((void**)&kt.stick_g0, kt.h_g0.data(), sizeof(int) * kt.h_g0.size())) ||
            (st = upload((void**)&kt.stick_plane, kt.h_plane.data(), sizeof(int) * kt.h_plane.size())) ||
            (st = upload((void**)&kt.rows, kt.h_rows.data(), sizeof(int) * kt.h_rows.size())) ||
            (st = upload((void**)&kt.g_code, kt.h_code.data(), sizeof(int2) * kt.h_code.size())) ||
            (st = upload((void**)&kt.kin, kt.h_kin.data(), sizeof(double) * kt.h_kin.size())) ||
            (st = upload((void**)&kt.kin_f, kinf.data(), sizeof(float) * kinf.size())))
            return st;
        if (kt.gamma && (st = upload((void**)&kt.gtile, kt.h_gtile.data(), sizeof(int2) * kt.h_gtile.size())))
            return st;
    }
    if ((st = cuda_check(cudaStreamCreateWithFlags(&g->aux, cudaStreamNonBlocking), "gspace stream")) ||
        (st = cuda_check(cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming), "gspace event")) ||
        (st = cuda_check(cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming), "gspace event")))
        return st;
    return QM_OK;
}

qm_status gspace_clone(qm_gspace g, qm_gspace* out) {
    qm_status st = ensure_device(g);
    if (st) return st;
    qm_gspace c = new (std::nothrow) qm_gspace_s(*g);
    if (!c) return fail(QM_ERR_OOM, "gspace clone: host allocation");
    c->ws = Workspace{};
    c->dws = Workspace{};
    c->prep.assign(c->nk, NlPrep{});  // prepared projectors belong to the origin
    c->aux = nullptr;
    c->ev_fork = c->ev_join = nullptr;
    c->shared_tables = true;
    if ((st = cuda_check(cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking), "gspace stream")) ||
        (st = cuda_check(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming), "gspace event")) ||
        (st = cuda_check(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming), "gspace event"))) {
        qm_gspace_destroy(c);
        return st;
    }
    *out = c;
    return QM_OK;
}

}  // namespace qm

using namespace qm;

extern "C" const char* qm_last_error(void) { return g_last_error.c_str(); }
extern "C" const char* qm_version(void) { return "qm-gb300 0.1 (sm_103a)"; }

extern "C" qm_status qm_gspace_create(const double lattice[9], int nk, const double* kpts,
                                      double ecutwfc_ha, const int grid_override[3],
                                      qm_gspace* out) {
    clear_error();
    if (!lattice || !kpts || !out) return fail(QM_ERR_ARG, "qm_gspace_create: NULL argument");
    *out = nullptr;
    if (nk < 1 || nk > 4096) return fail(QM_ERR_ARG, "qm_gspace_create: nk out of range");
    if (!(ecutwfc_ha > 0.0) || !std::isfinite(ecutwfc_ha))
        return fail(QM_ERR_ARG, "qm_gspace_create: ecutwfc_ha must be > 0");
    for (int i = 0; i < 9; ++i)
        if (!std::isfinite(lattice[i])) return fail(QM_ERR_ARG, "qm_gspace_create: non-finite lattice");

    auto* g = new qm_gspace_s();
    std::memcpy(g->lattice, lattice, sizeof(double) * 9);
    inv3_transpose_2pi(lattice, g->recip);
    double vol = std::fabs(lattice[0] * (lattice[4] * lattice[8] - lattice[5] * lattice[7]) -
                           lattice[1] * (lattice[3] * lattice[8] - lattice[5] * lattice[6]) +
                           lattice[2] * (lattice[3] * lattice[7] - lattice[4] * lattice[6]));
    if (!(vol > 1e-8)) {
        delete g;
        return fail(QM_ERR_ARG, "qm_gspace_create: singular lattice");
    }
    g->ecut = ecutwfc_ha;
    g->nk = nk;
    g->kpts.assign(kpts, kpts + 3 * nk);
    const double qmax = std::sqrt(2.0 * ecutwfc_ha);
    for (int d = 0; d < 3; ++d) {
        double alen = std::sqrt(lattice[3 * d] * lattice[3 * d] + lattice[3 * d + 1] * lattice[3 * d + 1] +
                                lattice[3 * d + 2] * lattice[3 * d + 2]);
        if (grid_override) {
            g->n[d] = grid_override[d];
            if (g->n[d] < 2 || g->n[d] > 512 || !smooth235(g->n[d])) {
                delete g;
                return fail(QM_ERR_ARG, "qm_gspace_create: grid_override must be 2,3,5-smooth in [2,512]");
            }
        } else {
            // dual cutoff: |G| <= 2 qmax  =>  n = floor(2 qmax |a| / 2 pi)
            int n = (int)std::floor(2.0 * qmax * alen / (2.0 * M_PI));
            int N = 2 * n + 1;
            while (!smooth235(N)) ++N;
            if (N > 512) {
                delete g;
                return fail(QM_ERR_ARG, "qm_gspace_create: grid rule gives N > 512");
            }
            g->n[d] = N;
        }
    }
    const int N1 = g->n[0], N2 = g->n[1], N3 = g->n[2];
    g->ldx = (N1 % 2 == 0) ? N1 + 1 : N1;
    g->ldy = (N2 % 2 == 0) ? N2 + 1 : N2;

    qm_status st = QM_OK;
    // FFT plans, twiddles exp(+2 pi i t / N) (quarter turns exact), digit-reversal tables
    for (int d = 0; d < 3; ++d) {
        fft_plan(g->n[d], 0, g->plan[d], g->h_rev[d]);
        int N = g->n[d];
        g->h_tw[d].resize(N);
        for (int t = 0; t < N; ++t) {
            double ang = 2.0 * M_PI * (double)t / (double)N;
            double c = std::cos(ang), sn = std::sin(ang);
            if ((4 * t) % N == 0) {
                int q = (4 * t) / N;
                c = (q == 0) ? 1.0 : (q == 2 ? -1.0 : 0.0);
                sn = (q == 1) ? 1.0 : (q == 3 ? -1.0 : 0.0);
            }
            g->h_tw[d][t] = make_double2(c, sn);
        }
    }

    // plane-wave spheres
    const double* b = g->recip;
    g->k.resize(nk);
    for (int ik = 0; ik < nk; ++ik) {
        const double* kc = kpts + 3 * ik;
        int lo[3], hi[3];
        for (int d = 0; d < 3; ++d) {
            double alen = std::sqrt(lattice[3 * d] * lattice[3 * d] + lattice[3 * d + 1] * lattice[3 * d + 1] +
                                    lattice[3 * d + 2] * lattice[3 * d + 2]);
            double bound = qmax * alen / (2.0 * M_PI);
            lo[d] = (int)std::floor(-kc[d] - bound) - 1;
            hi[d] = (int)std::ceil(-kc[d] + bound) + 1;
        }
        std::vector<PW> pws;
        for (int m3 = lo[2]; m3 <= hi[2]; ++m3)
            for (int m2 = lo[1]; m2 <= hi[1]; ++m2)
                for (int m1 = lo[0]; m1 <= hi[0]; ++m1) {
                    double c1 = m1 + kc[0], c2 = m2 + kc[1], c3 = m3 + kc[2];
                    PW p;
                    for (int x = 0; x < 3; ++x) p.q[x] = c1 * b[x] + c2 * b[3 + x] + c3 * b[6 + x];
                    p.kin = 0.5 * (p.q[0] * p.q[0] + p.q[1] * p.q[1] + p.q[2] * p.q[2]);
                    if (!(p.kin <= ecutwfc_ha * (1.0 + 1e-12))) continue;
                    p.m[0] = m1; p.m[1] = m2; p.m[2] = m3;
                    int i1 = ((m1 % N1) + N1) % N1, i2 = ((m2 % N2) + N2) % N2, i3 = ((m3 % N3) + N3) % N3;
                    p.idx = (int64_t)i1 + (int64_t)N1 * ((int64_t)i2 + (int64_t)N2 * i3);
                    pws.push_back(p);
                }
        std::sort(pws.begin(), pws.end(), [](const PW& x, const PW& y) { return x.idx < y.idx; });
        for (size_t i = 1; i < pws.size(); ++i)
            if (pws[i].idx == pws[i - 1].idx) {
                qm_gspace_destroy(g);
                return fail(QM_ERR_ARG, "qm_gspace_create: FFT grid too small for the plane-wave sphere");
            }
        KTables& kt = g->k[ik];
        kt.npw = (int)pws.size();
        if (kt.npw == 0) {
            qm_gspace_destroy(g);
            return fail(QM_ERR_ARG, "qm_gspace_create: empty plane-wave sphere");
        }
        // sticks along x: consecutive plane waves sharing (i2, i3)
        std::vector<int> g0, plane, rows;
        std::vector<int2> code(kt.npw);
        std::vector<double> kin(kt.npw);
        int64_t last = -1;
        for (int i = 0; i < kt.npw; ++i) {
            int64_t key = pws[i].idx / N1;
            if (key != last) {
                g0.push_back(i);
                int i2 = (int)(key % N2), i3 = (int)(key / N2);
                plane.push_back(i3 * g->ldy + i2);
                if (rows.empty() || rows.back() != i3) rows.push_back(i3);
                last = key;
            }
            code[i] = make_int2((int)g0.size() - 1, (int)(pws[i].idx % N1));
            kin[i] = pws[i].kin;
        }
        kt.nstick = (int)g0.size();
        g0.push_back(kt.npw);
        kt.nstick_pad = (int)align_up(kt.nstick, 4);
        std::sort(rows.begin(), rows.end());
        rows.erase(std::unique(rows.begin(), rows.end()), rows.end());
        kt.nrow = (int)rows.size();
        kt.h_idx.resize(kt.npw);
        kt.h_miller.resize(3 * (size_t)kt.npw);
        kt.h_kpg.resize(3 * (size_t)kt.npw);
        for (int i = 0; i < kt.npw; ++i) {
            kt.h_idx[i] = (int32_t)pws[i].idx;
            for (int x = 0; x < 3; ++x) {
                kt.h_miller[3 * i + x] = pws[i].m[x];
                kt.h_kpg[3 * i + x] = pws[i].q[x];
            }
        }
        if (kc[0] == 0.0 && kc[1] == 0.0 && kc[2] == 0.0) {
            // Gamma point: pair every stick (i2, i3) with the stick (-i2, -i3) that holds the -G of
            // its plane waves (the sphere is symmetric under G -> -G at k = 0); pairs fill slots
            // j and j + kGammaTile/2 of a tile, sticks that are their own partner (i2, i3 each 0
            // or N/2) get tiles of their own
            const int half = kGammaTile / 2;
            std::vector<int> partner(kt.nstick, -1);
            std::vector<int64_t> keys(kt.nstick);
            for (int s2 = 0; s2 < kt.nstick; ++s2) keys[s2] = (int64_t)pws[g0[s2]].idx / N1;
            bool ok = true;
            for (int s2 = 0; s2 < kt.nstick && ok; ++s2) {
                const int i2 = (int)(keys[s2] % N2), i3 = (int)(keys[s2] / N2);
                const int64_t pk = (int64_t)((N2 - i2) % N2) + (int64_t)N2 * ((N3 - i3) % N3);
                auto it = std::lower_bound(keys.begin(), keys.end(), pk);
                if (it == keys.end() || *it != pk) ok = false;
                else partner[s2] = (int)(it - keys.begin());
            }
            if (ok) {
                std::vector<int2> tiles, self_tiles;
                int np = 0, nself = 0;
                for (int s2 = 0; s2 < kt.nstick; ++s2) {
                    const int p2 = partner[s2];
                    if (p2 == s2) {
                        if (nself % kGammaTile == 0) self_tiles.resize(self_tiles.size() + kGammaTile, make_int2(-1, 0));
                        const int slot = nself % kGammaTile;
                        self_tiles[self_tiles.size() - kGammaTile + slot] = make_int2(s2, slot);
                        ++nself;
                    } else if (p2 > s2) {
                        if (np % half == 0) tiles.resize(tiles.size() + kGammaTile, make_int2(-1, 0));
                        const int slot = np % half;
                        tiles[tiles.size() - kGammaTile + slot] = make_int2(s2, slot + half);
                        tiles[tiles.size() - kGammaTile + slot + half] = make_int2(p2, slot);
                        ++np;
                    }
                }
                tiles.insert(tiles.end(), self_tiles.begin(), self_tiles.end());
                kt.gamma = true;
                kt.ngtile = (int)(tiles.size() / kGammaTile);
                kt.h_gtile = std::move(tiles);
            }
        }
        kt.h_g0 = std::move(g0);
        kt.h_plane = std::move(plane);
        kt.h_rows = std::move(rows);
        kt.h_code = std::move(code);
        kt.h_kin = std::move(kin);
    }
    *out = g;
    return QM_OK;
}

extern "C" qm_status qm_gspace_query(qm_gspace g, int grid[3], int* npw, int* npw_max, int* nk) {
    clear_error();
    if (!g) return fail(QM_ERR_ARG, "qm_gspace_query: NULL handle");
    if (grid) for (int d = 0; d < 3; ++d) grid[d] = g->n[d];
    int mx = 0;
    for (int ik = 0; ik < g->nk; ++ik) {
        if (npw) npw[ik] = g->k[ik].npw;
        mx = std::max(mx, g->k[ik].npw);
    }
    if (npw_max) *npw_max = mx;
    if (nk) *nk = g->nk;
    return QM_OK;
}

extern "C" qm_status qm_gspace_indices(qm_gspace g, int ik, int32_t* idx, int32_t* miller, double* kpg) {
    clear_error();
    if (!g) return fail(QM_ERR_ARG, "qm_gspace_indices: NULL handle");
    if (ik < 0 || ik >= g->nk) return fail(QM_ERR_ARG, "qm_gspace_indices: ik out of range");
    const KTables& kt = g->k[ik];
    if (idx) std::memcpy(idx, kt.h_idx.data(), sizeof(int32_t) * kt.npw);
    if (miller) std::memcpy(miller, kt.h_miller.data(), sizeof(int32_t) * 3 * (size_t)kt.npw);
    if (kpg) std::memcpy(kpg, kt.h_kpg.data(), sizeof(double) * 3 * (size_t)kt.npw);
    return QM_OK;
}

extern "C" qm_status qm_gspace_sticks(qm_gspace g, int ik, int* nstick, int32_t* stick_yz, int* ngtile,
                                      int32_t* gtile) {
    clear_error();
    if (!g) return fail(QM_ERR_ARG, "qm_gspace_sticks: NULL handle");
    if (ik < 0 || ik >= g->nk) return fail(QM_ERR_ARG, "qm_gspace_sticks: ik out of range");
    const KTables& kt = g->k[ik];
    const int N2 = g->n[1];
    if (nstick) *nstick = kt.nstick;
    if (ngtile) *ngtile = kt.gamma ? kt.ngtile : 0;
    if (stick_yz)
        for (int s = 0; s < kt.nstick; ++s) {
            const int64_t key = (int64_t)kt.h_idx[kt.h_g0[s]] / g->n[0];
            stick_yz[2 * s] = (int32_t)(key % N2);
            stick_yz[2 * s + 1] = (int32_t)(key / N2);
        }
    if (gtile && kt.gamma)
        for (size_t i = 0; i < kt.h_gtile.size(); ++i) {
            gtile[2 * i] = kt.h_gtile[i].x;
            gtile[2 * i + 1] = kt.h_gtile[i].y;
        }
    return QM_OK;
}

extern "C" void qm_gspace_destroy(qm_gspace g) {
    if (!g) return;
    if (g->uploaded) {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(g->device);
        cudaDeviceSynchronize();
        for (auto& kt : g->k) {
            if (g->shared_tables) break;
            cudaFree(kt.stick_g0);
            cudaFree(kt.stick_plane);
            cudaFree(kt.rows);
            cudaFree(kt.g_code);
            cudaFree(kt.kin);
            cudaFree(kt.kin_f);
            cudaFree(kt.gtile);
        }
        for (int d = 0; d < 3 && !g->shared_tables; ++d) {
            cudaFree(g->tw64[d]);
            cudaFree(g->tw32[d]);
            cudaFree(g->rev[d]);
        }
        if (g->ws.ptr) cudaFree(g->ws.ptr);
        if (g->dws.ptr) cudaFree(g->dws.ptr);
        for (auto& p : g->prep)
            if (p.dev) cudaFree(p.dev);
        if (g->ev_fork) cudaEventDestroy(g->ev_fork);
        if (g->ev_join) cudaEventDestroy(g->ev_join);
        if (g->aux) cudaStreamDestroy(g->aux);
        cudaSetDevice(cur);
    }
    delete g;
}
