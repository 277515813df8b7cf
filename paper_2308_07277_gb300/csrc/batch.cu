// Host side of the batched H psi (batch.cuh): work-item lists, device layout, CUDA-graph
// capture of the one persistent launch, and the autotuner that picks its shape.
#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <numeric>
#include <utility>
#include <vector>

#include "batch.cuh"

namespace qm {
qm_status batch_launch_f32(const BatchLaunch& L, cudaStream_t s);
qm_status batch_launch_f64(const BatchLaunch& L, cudaStream_t s);
int batch_occupancy_f32(size_t smem, int order);
int batch_occupancy_f64(size_t smem, int order);
}  // namespace qm

using namespace qm;

struct qm_batch_s {
    int device = 0;
    qm_precision prec = QM_FP64;
    std::vector<qm_hpsi_job> jobs;
    int ctas = 0, points = 0, group_mb = 0, grid = 0, nitems = 0, ncells = 0, candidates = 0;
    int order = 0;  // FFT radix order of the built plan
    size_t smem = 0, dbytes = 0;
    double tuned_ms = 0.0;
    long long band_applies = 0;
    void* dmem = nullptr;
    int* err = nullptr;
    BatchCtl* ctl = nullptr;  // device controls of the bounded waits
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;
};

namespace {

constexpr int kCandCtas[] = {1, 2, 3, 4};
constexpr int kCandPoints[] = {1024, 2048, 4096, 8192};
constexpr int kCandGroupMb[] = {24, 48, -1};  // tried at the best (ctas, points) of the first: -1 = one group

struct Region {
    size_t off = 0;
    size_t take(size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    }
};

void release(qm_batch b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    if (b->dmem) cudaFree(b->dmem);
    b->dmem = nullptr;
    b->err = nullptr;
}

// Build the work lists and device data for one shape and capture the launch in a graph.
// `infeasible` is set (and QM_OK returned) when the shape does not fit the SM.
qm_status build(qm_batch b, int ctas, int points, size_t group_bytes, int radix_order, bool* infeasible) {
    *infeasible = false;
    const bool fp32 = b->prec == QM_MIXED;
    const size_t cs = fp32 ? sizeof(float2) : sizeof(double2);
    const size_t rs = fp32 ? sizeof(float) : sizeof(double);
    const int nj = (int)b->jobs.size();

    // distinct (gspace, V) pairs share one V layout
    std::map<std::pair<const void*, const void*>, int> cell_of;
    std::vector<int> job_cell(nj);
    std::vector<const qm_hpsi_job*> cell_job;
    for (int j = 0; j < nj; ++j) {
        const auto key = std::make_pair((const void*)b->jobs[j].g, (const void*)b->jobs[j].vloc_r);
        auto it = cell_of.find(key);
        if (it == cell_of.end()) {
            it = cell_of.emplace(key, (int)cell_job.size()).first;
            cell_job.push_back(&b->jobs[j]);
        }
        job_cell[j] = it->second;
    }
    const int nc = (int)cell_job.size();

    std::vector<BatchJobDev> J(nj);
    std::vector<BatchCellDev> Cl(nc);
    // the FFT plans (and digit-reversal tables) of every length in the chosen radix order
    std::map<int, std::pair<AxisPlan, std::vector<int>>> plans;
    auto plan_of = [&](int n) -> const std::pair<AxisPlan, std::vector<int>>& {
        auto it = plans.find(n);
        if (it == plans.end()) {
            it = plans.emplace(n, std::make_pair(AxisPlan{}, std::vector<int>())).first;
            fft_plan(n, radix_order, it->second.first, it->second.second);
        }
        return it->second;
    };
    size_t smem = (size_t)kBatchAB * kBatchAP * cs;  // application staging
    for (int j = 0; j < nj; ++j) {
        const qm_hpsi_job& q = b->jobs[j];
        const qm_gspace g = q.g;
        const KTables& kt = g->k[q.ik];
        BatchJobDev& d = J[j];
        std::memset(&d, 0, sizeof(d));
        d.n1 = g->n[0];
        d.n2 = g->n[1];
        d.n3 = g->n[2];
        d.ldx = g->ldx;
        d.ldy = g->ldy;
        d.nstick = kt.nstick;
        d.nstick_pad = kt.nstick_pad;
        d.nrow = kt.nrow;
        d.npw = kt.npw;
        d.nb = q.nb;
        d.nproj = q.nproj;
        d.nl = std::max(4, std::min(256, points / d.n1));
        d.nk1 = (d.nb * d.nstick + d.nl - 1) / d.nl;
        d.bpp = std::max(1, std::min(std::min(8, d.nb), points / (d.n2 * d.n3)));
        d.nk2 = d.n1 * ((d.nb + d.bpp - 1) / d.bpp);
        d.nchunk = (d.npw + kBatchGC - 1) / kBatchGC;
        if (d.nproj > 0) {
            const int npt = (d.nproj + 3) / 4;
            if (npt > kThreads) return fail(QM_ERR_UNSUPPORTED, "batched H psi: more than 1024 projectors");
            d.bblk = std::min(d.nb, 4 * (kThreads / npt));
            d.nbblk = (d.nb + d.bblk - 1) / d.bblk;
            d.nnla = (d.npw + kBatchGA - 1) / kBatchGA;
            smem = std::max(smem, (size_t)kBatchSG * (npt * 4 + ((d.bblk + 3) / 4) * 4) * cs);
        }
        d.cell = job_cell[j];
        d.ld_psi = q.ld_psi;
        d.ld_out = q.ld_out;
        d.ld_beta = q.ld_beta;
        d.px = plan_of(g->n[0]).first;
        d.py = plan_of(g->n[1]).first;
        d.pz = plan_of(g->n[2]).first;
        d.stick_g0 = kt.stick_g0;
        d.stick_plane = kt.stick_plane;
        d.g_code = kt.g_code;
        d.kin = fp32 ? (const void*)kt.kin_f : (const void*)kt.kin;
        for (int a = 0; a < 3; ++a) d.tw[a] = fp32 ? (const void*)g->tw32[a] : (const void*)g->tw64[a];
        d.psi = q.psi;
        d.out = q.out;
        d.beta = q.beta;
        d.D = q.D;
        smem = std::max(smem, (size_t)(d.nl * d.ldx + d.n1) * cs);
        smem = std::max(smem, (size_t)(d.bpp * d.n3 * d.ldy + d.n2 + d.n3) * cs);
    }
    if (smem > 227 * 1024) {
        *infeasible = true;
        return QM_OK;
    }
    const int occ = fp32 ? batch_occupancy_f32(smem, radix_order) : batch_occupancy_f64(smem, radix_order);
    if (occ < ctas) {
        *infeasible = true;
        return QM_OK;
    }

    // device layout
    Region R;
    const size_t o_ctl = R.take(sizeof(BatchCtl));
    const size_t o_jobs = R.take(sizeof(BatchJobDev) * nj);
    const size_t o_cells = R.take(sizeof(BatchCellDev) * nc);
    std::vector<int4> items;
    const size_t n_cnt = (size_t)nj * kBatchCounters + nc + 2;
    std::vector<size_t> o_rows(nj), o_cols(nj), o_T(nj), o_part(nj), o_Pd(nj), o_vt(nc);
    // Item list.  Jobs (largest first) are cut into groups whose stick buffers hold at most
    // `group_bytes` (0: one group); the phases of consecutive groups are interleaved as a
    // software pipeline, stage t = [NLA of group t-3, K3 of t-2, NLR + K2 of t-1, VT + NLP +
    // K1 of t], so only the stick buffers of about three groups are live at a time (they stay
    // in L2) and every item still depends only on items of earlier tickets.
    std::vector<int> order(nj);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        const double wa = (double)J[a].nb * J[a].n1 * J[a].n2 * J[a].n3;
        const double wc = (double)J[c].nb * J[c].n1 * J[c].n2 * J[c].n3;
        return wa > wc;
    });
    std::vector<std::vector<int>> groups(1);
    {
        size_t acc = 0;
        for (int j : order) {
            const size_t tb = cs * (size_t)J[j].nb * J[j].n1 * J[j].nstick_pad;
            if (group_bytes > 0 && !groups.back().empty() && acc + tb > group_bytes) {
                groups.emplace_back();
                acc = 0;
            }
            groups.back().push_back(j);
            acc += tb;
        }
    }
    for (int c = 0; c < nc; ++c) {
        const qm_gspace g = cell_job[c]->g;
        const long long nr = (long long)g->n[0] * g->n[1] * g->n[2];
        Cl[c].nchunk = (int)((nr + kBatchVTC - 1) / kBatchVTC);
    }
    std::vector<char> vt_done(nc, 0);
    const int ng = (int)groups.size();
    for (int t = 0; t < ng + 3; ++t) {
        if (t - 3 >= 0 && t - 3 < ng)
            for (int j : groups[t - 3])
                if (J[j].nproj > 0)
                    for (int q = 0; q < J[j].nnla; ++q) items.push_back(make_int4(BK_NLA, j, q, 0));
        if (t - 2 >= 0 && t - 2 < ng)
            for (int j : groups[t - 2])
                for (int q = 0; q < J[j].nk1; ++q) items.push_back(make_int4(BK_K3, j, q, 0));
        if (t - 1 >= 0 && t - 1 < ng)
            for (int j : groups[t - 1]) {
                if (J[j].nproj > 0) items.push_back(make_int4(BK_NLR, j, 0, 0));
                const int ngrp = (J[j].nb + J[j].bpp - 1) / J[j].bpp;
                for (int p1 = 0; p1 < J[j].n1; ++p1)
                    for (int gr = 0; gr < ngrp; ++gr) items.push_back(make_int4(BK_K2, j, gr, p1));
            }
        if (t < ng) {
            for (int j : groups[t]) {
                const int c = J[j].cell;
                if (!vt_done[c]) {
                    vt_done[c] = 1;
                    for (int k = 0; k < Cl[c].nchunk; ++k) items.push_back(make_int4(BK_VT, c, k, 0));
                }
            }
            for (int j : groups[t])
                if (J[j].nproj > 0)
                    for (int ch = 0; ch < J[j].nchunk; ++ch)
                        for (int bb = 0; bb < J[j].nbblk; ++bb) items.push_back(make_int4(BK_NLP, j, ch, bb));
            for (int j : groups[t])
                for (int q = 0; q < J[j].nk1; ++q) items.push_back(make_int4(BK_K1, j, q, 0));
        }
    }
    const size_t o_items = R.take(sizeof(int4) * items.size());
    const size_t o_cnt = R.take(sizeof(int) * n_cnt);
    for (int j = 0; j < nj; ++j) {
        o_rows[j] = R.take(sizeof(int) * (size_t)J[j].bpp * J[j].nrow);
        o_cols[j] = R.take(sizeof(int) * (size_t)J[j].bpp * J[j].n2);
    }
    // digit-reversal tables of the radix order 1 plans (order 0 uses the gspace's own)
    std::map<int, size_t> o_rev;
    if (radix_order)
        for (int c = 0; c < nc; ++c)
            for (int a = 0; a < 3; ++a) {
                const int n = cell_job[c]->g->n[a];
                if (!o_rev.count(n)) o_rev[n] = R.take(sizeof(int) * (size_t)n);
            }
    const size_t table_end = R.off;
    for (int c = 0; c < nc; ++c) {
        const qm_gspace g = cell_job[c]->g;
        o_vt[c] = R.take(rs * (size_t)g->n[0] * g->n[1] * g->n[2]);
    }
    for (int j = 0; j < nj; ++j) {
        o_T[j] = R.take(cs * (size_t)J[j].nb * J[j].n1 * J[j].nstick_pad);
        o_part[j] = R.take(cs * (size_t)J[j].nchunk * J[j].nb * J[j].nproj);
        o_Pd[j] = R.take(cs * (size_t)J[j].nb * J[j].nproj);
    }
    const size_t total = R.off;

    void* dmem = nullptr;
    qm_status st = cuda_check(cudaMalloc(&dmem, total), "batched H psi: cudaMalloc");
    if (st) return st == QM_ERR_CUDA ? fail(QM_ERR_OOM, "batched H psi: device allocation failed") : st;
    char* base = (char*)dmem;
    std::vector<char> img(table_end, 0);
    for (int j = 0; j < nj; ++j) {
        const qm_hpsi_job& q = b->jobs[j];
        const KTables& kt = q.g->k[q.ik];
        BatchJobDev& d = J[j];
        d.rows2 = (const int*)(base + o_rows[j]);
        d.cols2 = (const int*)(base + o_cols[j]);
        d.T = base + o_T[j];
        d.part = base + o_part[j];
        d.Pd = base + o_Pd[j];
        int* rows2 = (int*)(img.data() + o_rows[j]);
        for (int l = 0; l < d.bpp * d.nrow; ++l) rows2[l] = (l / d.nrow) * d.n3 + kt.h_rows[l % d.nrow];
        int* cols2 = (int*)(img.data() + o_cols[j]);
        for (int l = 0; l < d.bpp * d.n2; ++l) cols2[l] = (l / d.n2) * d.n3 * d.ldy + l % d.n2;
    }
    for (int c = 0; c < nc; ++c) {
        const qm_gspace g = cell_job[c]->g;
        Cl[c].V = cell_job[c]->vloc_r;
        Cl[c].vt = base + o_vt[c];
        Cl[c].n1 = g->n[0];
        Cl[c].n2 = g->n[1];
        Cl[c].n3 = g->n[2];
        for (int a = 0; a < 3; ++a)
            Cl[c].rev[a] = radix_order ? (const int*)(base + o_rev[g->n[a]]) : g->rev[a];
        Cl[c].scale = 1.0 / ((double)g->n[0] * g->n[1] * g->n[2]);
    }
    {
        const BatchCtl ctl{kBatchSpinLimit, -1, 0};
        std::memcpy(img.data() + o_ctl, &ctl, sizeof(ctl));
    }
    for (const auto& kv : o_rev) {
        const std::vector<int>& rv = plan_of(kv.first).second;
        std::memcpy(img.data() + kv.second, rv.data(), sizeof(int) * rv.size());
    }
    std::memcpy(img.data() + o_jobs, J.data(), sizeof(BatchJobDev) * nj);
    std::memcpy(img.data() + o_cells, Cl.data(), sizeof(BatchCellDev) * nc);
    std::memcpy(img.data() + o_items, items.data(), sizeof(int4) * items.size());
    st = cuda_check(cudaMemcpy(dmem, img.data(), table_end, cudaMemcpyHostToDevice), "batched H psi: upload");
    if (st) {
        cudaFree(dmem);
        return st;
    }

    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device);
    BatchLaunch L{};
    L.ctl = (const BatchCtl*)(base + o_ctl);
    L.jobs = (const BatchJobDev*)(base + o_jobs);
    L.cells = (const BatchCellDev*)(base + o_cells);
    L.items = (const int4*)(base + o_items);
    L.nitems = (int)items.size();
    L.cnt = (int*)(base + o_cnt);
    L.cell_cnt = L.cnt + (size_t)nj * kBatchCounters;
    L.head = L.cell_cnt + nc;
    L.err = L.head + 1;
    L.order = radix_order;
    L.grid = std::max(1, std::min(ctas * nsm, L.nitems));
    L.smem = smem;

    // capture: reset the counters, ticket and error word, then the persistent launch
    if (!b->cap) {
        st = cuda_check(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking), "batched H psi: stream");
        if (st) {
            cudaFree(dmem);
            return st;
        }
    }
    cudaGraph_t graph = nullptr;
    st = cuda_check(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "batched H psi: capture");
    if (!st) {
        cudaMemsetAsync(L.cnt, 0, sizeof(int) * n_cnt, b->cap);
        const qm_status sl = fp32 ? batch_launch_f32(L, b->cap) : batch_launch_f64(L, b->cap);
        st = cuda_check(cudaStreamEndCapture(b->cap, &graph), "batched H psi: end capture");
        if (!st && sl) st = sl;
    }
    cudaGraphExec_t exec = nullptr;
    if (!st) st = cuda_check(cudaGraphInstantiate(&exec, graph, 0), "batched H psi: graph instantiate");
    if (graph) cudaGraphDestroy(graph);
    if (st) {
        cudaFree(dmem);
        return st;
    }
    b->dmem = dmem;
    b->exec = exec;
    b->err = L.err;
    b->ctl = (BatchCtl*)(base + o_ctl);
    b->ctas = ctas;
    b->points = points;
    b->group_mb = group_bytes ? (int)(group_bytes >> 20) : -1;
    b->grid = L.grid;
    b->nitems = L.nitems;
    b->ncells = nc;
    b->smem = smem;
    b->dbytes = total;
    b->order = radix_order;
    return QM_OK;
}

qm_status launch(qm_batch b, cudaStream_t s) {
    ProfScope pf(PF_BATCH, s);
    return cuda_check(cudaGraphLaunch(b->exec, s), "batched H psi: graph launch");
}

qm_status read_err(qm_batch b, cudaStream_t s) {
    int e = 0;
    qm_status st = cuda_check(cudaStreamSynchronize(s), "batched H psi: synchronize");
    if (st) return st;
    if ((st = cuda_check(cudaMemcpy(&e, b->err, sizeof(int), cudaMemcpyDeviceToHost), "batched H psi: error word")))
        return st;
    return e ? fail(QM_ERR_TIMEOUT, "batched H psi: a bounded device-side wait expired") : QM_OK;
}

// median of `reps` timed runs (after one warm-up run) in ms
qm_status time_runs(qm_batch b, cudaStream_t s, int reps, double* ms) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::vector<double> t;
    qm_status st = launch(b, s);
    for (int r = 0; r < reps && !st; ++r) {
        cudaEventRecord(e0, s);
        st = launch(b, s);
        cudaEventRecord(e1, s);
        if (!st) st = cuda_check(cudaEventSynchronize(e1), "batched H psi: tuner sync");
        float x = 0.f;
        if (!st) cudaEventElapsedTime(&x, e0, e1);
        t.push_back(x);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!st) st = read_err(b, s);
    if (st) return st;
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return QM_OK;
}

qm_status check_job(const qm_hpsi_job& q, bool fp32, int i) {
    const std::string w = "qm_batch_create: job " + std::to_string(i) + ": ";
    if (!q.g) return fail(QM_ERR_ARG, w + "NULL gspace");
    if (q.ik < 0 || q.ik >= q.g->nk) return fail(QM_ERR_ARG, w + "ik out of range");
    if (q.nb < 1 || q.nproj < 0) return fail(QM_ERR_ARG, w + "nb < 1 or nproj < 0");
    const int npw = q.g->k[q.ik].npw;
    if (!q.psi || !q.out || !q.vloc_r) return fail(QM_ERR_ARG, w + "NULL psi, out or vloc_r");
    if (q.ld_psi < npw || q.ld_out < npw) return fail(QM_ERR_ARG, w + "leading dimension < npw");
    if (q.nproj > 0 && (!q.beta || !q.D || q.ld_beta < npw)) return fail(QM_ERR_ARG, w + "beta, D or ld_beta");
    const uintptr_t al = fp32 ? 8 : 16;
    if (((uintptr_t)q.psi | (uintptr_t)q.out | (q.nproj > 0 ? (uintptr_t)q.beta : 0)) % al)
        return fail(QM_ERR_ARG, w + "psi/out/beta not aligned to the complex element size");
    const size_t cs = fp32 ? sizeof(float2) : sizeof(double2);
    const char* a0 = (const char*)q.psi;
    const char* a1 = a0 + ((size_t)(q.nb - 1) * q.ld_psi + npw) * cs;
    const char* b0 = (const char*)q.out;
    const char* b1 = b0 + ((size_t)(q.nb - 1) * q.ld_out + npw) * cs;
    if (a0 < b1 && b0 < a1) return fail(QM_ERR_ARG, w + "out overlaps psi");
    return QM_OK;
}

}  // namespace

extern "C" qm_status qm_batch_create(int njobs, const qm_hpsi_job* jobs, qm_precision prec,
                                     const qm_batch_shape* shape, void* stream, qm_batch* out) {
    clear_error();
    if (!out) return fail(QM_ERR_ARG, "qm_batch_create: NULL out");
    *out = nullptr;
    if (njobs < 1 || !jobs) return fail(QM_ERR_ARG, "qm_batch_create: no jobs");
    if (prec != QM_FP64 && prec != QM_MIXED) return fail(QM_ERR_ARG, "qm_batch_create: unknown precision");
    const bool fp32 = prec == QM_MIXED;
    int ctas = shape ? shape->ctas_per_sm : 0, points = shape ? shape->item_points : 0;
    int gmb = shape ? shape->group_mb : 0;
    const int ford = shape ? shape->fft_order : 0;  // 0: autotune; 1, 2: radix order 0, 1
    if (ctas < 0 || ctas > 8 || points < 0 || (points > 0 && (points < 256 || points > 65536)) || gmb < -1 ||
        gmb > 4096 || ford < 0 || ford > 2)
        return fail(QM_ERR_ARG, "qm_batch_create: shape out of range");
    auto gbytes = [](int mb) { return mb > 0 ? (size_t)mb << 20 : (size_t)0; };
    qm_status st;
    for (int i = 0; i < njobs; ++i)
        if ((st = check_job(jobs[i], fp32, i))) return st;
    {
        // outputs of different jobs must not overlap (each job writes its whole block)
        const size_t cs = fp32 ? sizeof(float2) : sizeof(double2);
        std::vector<std::pair<const char*, const char*>> spans(njobs);
        for (int i = 0; i < njobs; ++i) {
            const char* a = (const char*)jobs[i].out;
            spans[i] = {a, a + ((size_t)(jobs[i].nb - 1) * jobs[i].ld_out + jobs[i].g->k[jobs[i].ik].npw) * cs};
        }
        std::sort(spans.begin(), spans.end());
        for (int i = 1; i < njobs; ++i)
            if (spans[i].first < spans[i - 1].second) return fail(QM_ERR_ARG, "qm_batch_create: outputs of two jobs overlap");
    }
    qm_batch b = new (std::nothrow) qm_batch_s;
    if (!b) return fail(QM_ERR_OOM, "qm_batch_create: host allocation");
    b->prec = prec;
    b->jobs.assign(jobs, jobs + njobs);
    for (const auto& q : b->jobs) b->band_applies += q.nb;
    if ((st = cuda_check(cudaGetDevice(&b->device), "cudaGetDevice"))) {
        delete b;
        return st;
    }
    for (const auto& q : b->jobs)
        if ((st = ensure_device(q.g))) {
            delete b;
            return st;
        }
    cudaStream_t s = (cudaStream_t)stream;
    bool infeasible = false;
    if (ctas > 0 && points > 0 && gmb != 0 && ford != 0) {
        st = build(b, ctas, points, gbytes(gmb), ford - 1, &infeasible);
        if (!st && infeasible) st = fail(QM_ERR_UNSUPPORTED, "qm_batch_create: shape does not fit the SM");
    } else {
        // autotune (each timed run executes the whole batch): every feasible (CTAs per SM,
        // points per item) at the first group size and radix order 0, then the group sizes at
        // the best of those, then the other radix order at the best shape
        double best = 1e300;
        int bc = 0, bp = 0, bg = gmb != 0 ? gmb : kCandGroupMb[0];
        const int o0 = ford ? ford - 1 : 0;
        int bo = o0;
        st = QM_OK;
        auto try_shape = [&](int c, int p, int g, int o) -> qm_status {
            qm_status s2 = build(b, c, p, gbytes(g), o, &infeasible);
            if (s2 || infeasible) return s2;
            double ms = 0.0;
            s2 = time_runs(b, s, 3, &ms);
            release(b);
            if (s2) return s2;
            ++b->candidates;
            if (ms < best) {
                best = ms;
                bc = c;
                bp = p;
                bg = g;
                bo = o;
            }
            return QM_OK;
        };
        const int g0 = bg;
        for (int c : kCandCtas) {
            if (ctas > 0 && c != ctas) continue;
            for (int p : kCandPoints) {
                if (points > 0 && p != points) continue;
                if ((st = try_shape(c, p, g0, o0))) break;
            }
            if (st) break;
        }
        if (!st && bc != 0 && gmb == 0) {
            const int c = bc, p = bp;
            for (int g : kCandGroupMb)
                if (g != g0 && (st = try_shape(c, p, g, o0))) break;
        }
        if (!st && bc != 0 && ford == 0) st = try_shape(bc, bp, bg, 1 - o0);
        if (!st && bc == 0) st = fail(QM_ERR_UNSUPPORTED, "qm_batch_create: no shape fits the SM");
        if (!st) {
            const int cands = b->candidates;
            st = build(b, bc, bp, gbytes(bg), bo, &infeasible);
            b->candidates = cands;
            b->tuned_ms = best;
        }
    }
    if (st) {
        release(b);
        if (b->cap) cudaStreamDestroy(b->cap);
        delete b;
        return st;
    }
    *out = b;
    return QM_OK;
}

extern "C" qm_status qm_batch_run(qm_batch b, void* stream) {
    clear_error();
    if (!b || !b->exec) return fail(QM_ERR_ARG, "qm_batch_run: invalid batch");
    return launch(b, (cudaStream_t)stream);
}

extern "C" qm_status qm_batch_check(qm_batch b, void* stream) {
    clear_error();
    if (!b || !b->exec) return fail(QM_ERR_ARG, "qm_batch_check: invalid batch");
    return read_err(b, (cudaStream_t)stream);
}

extern "C" qm_status qm_batch_hold(qm_batch b, int job, long long spin_limit) {
    clear_error();
    if (!b || !b->exec || !b->ctl) return fail(QM_ERR_ARG, "qm_batch_hold: invalid batch");
    if (job < -1 || job >= (int)b->jobs.size()) return fail(QM_ERR_ARG, "qm_batch_hold: job out of range");
    if (spin_limit < 0) return fail(QM_ERR_ARG, "qm_batch_hold: negative spin_limit");
    const BatchCtl ctl{spin_limit > 0 ? spin_limit : kBatchSpinLimit, job, job >= 0 ? 1 : 0};
    qm_status st = cuda_check(cudaDeviceSynchronize(), "qm_batch_hold: synchronize");
    if (st) return st;
    return cuda_check(cudaMemcpy(b->ctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice), "qm_batch_hold: upload");
}

extern "C" qm_status qm_batch_query(qm_batch b, qm_batch_info* info) {
    clear_error();
    if (!b || !info) return fail(QM_ERR_ARG, "qm_batch_query: NULL argument");
    info->ctas_per_sm = b->ctas;
    info->item_points = b->points;
    info->group_mb = b->group_mb;
    info->grid = b->grid;
    info->items = b->nitems;
    info->cells = b->ncells;
    info->candidates = b->candidates;
    info->band_applies = b->band_applies;
    info->smem_bytes = (long long)b->smem;
    info->device_bytes = (long long)b->dbytes;
    info->tuned_ms = b->tuned_ms;
    info->fft_order = b->order;
    return QM_OK;
}

extern "C" void qm_batch_destroy(qm_batch b) {
    if (!b) return;
    cudaDeviceSynchronize();
    release(b);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}
