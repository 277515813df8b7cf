/*
 * qm.h - C ABI of the GB300 plane-wave H-psi / block-Davidson library.
 *
 * Physics follows the plane-wave Kohn-Sham Hamiltonian of arXiv:2308.07277
 * (Quantum MASALA):
 *   (H psi)(G) = 1/2 |k+G|^2 psi(G)                                  [Sec. 2.2, Eq. KSHamMat]
 *              + sum_{G'} Vt((G-G') mod N) psi(G')                    [Sec. 2.2 / Sec. 4.3]
 *              + sum_p beta_p(G) D_p sum_{G'} conj(beta_p(G')) psi(G') [Sec. 2.3, KB form]
 * where Vt(g) = (1/N_r) sum_j V(r_j) exp(-i g.r_j) on the FFT grid, i.e. exactly the
 * "inverse FFT -> multiply by V(r) -> forward FFT -> keep the sphere" recipe of Sec. 4.3
 * with the r2g convention fftn(f).take(idxgrid) of the GSpaceBase example (Sec. 4.3.2).
 *
 * Conventions shared by every call
 *  - Units: Hartree atomic units (bohr, Hartree).
 *  - Complex numbers are interleaved (re, im): double[2] in FP64, float[2] in FP32.
 *  - Real-space grids are flat with x fastest: r index = j1 + N1*(j2 + N2*j3).
 *  - The plane waves of k-point ik are ordered by their flat grid index
 *    i1 + N1*(i2 + N2*i3), i_d = m_d mod N_d (G_1 varies fastest, as the paper prints).
 *  - Wavefunction blocks are band-major: psi[b*ld + g], ld >= npw(ik).
 *  - "device" pointers are CUDA device (or managed) memory owned by the caller; the
 *    library never frees them.  "host" pointers are ordinary host memory.
 *  - No exception crosses the ABI.  Every call returns a qm_status; on failure
 *    qm_last_error() returns a thread-local, NUL-terminated message describing it.
 *  - Asynchronous calls are ordered on the CUDA stream passed as `stream`
 *    (a cudaStream_t, NULL = legacy default stream).  A gspace handle owns a device
 *    workspace: calls that share a handle must be issued on ONE stream (or be
 *    otherwise serialised); use one handle per concurrent stream.
 *  - The library never falls back to a CPU path: without a usable CUDA device every
 *    compute call returns QM_ERR_CUDA.
 */
#ifndef QM_H
#define QM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qm_gspace_s* qm_gspace;   /* opaque, library-owned */

typedef enum {
    QM_OK = 0,
    QM_ERR_ARG = 1,            /* invalid argument (NULL, size, range); nothing launched */
    QM_ERR_CUDA = 2,           /* a CUDA runtime call or launch failed */
    QM_ERR_OOM = 3,            /* device or host allocation failed */
    QM_ERR_NOT_CONVERGED = 4,  /* Davidson hit max_iter; outputs still written */
    QM_ERR_NUMERIC = 5,        /* non-finite value or breakdown (e.g. Cholesky) */
    QM_ERR_TIMEOUT = 6,        /* a bounded device-side wait expired */
    QM_ERR_UNSUPPORTED = 7     /* valid request the library does not implement */
} qm_status;

typedef enum {
    QM_FP64 = 0,   /* everything in FP64 */
    QM_MIXED = 1   /* FP32 FFT path and V multiply; nonlocal projection and application as
                      3-term BF16 split products on the tensor cores, FP32 accumulation */
} qm_precision;

/*
 * qm_gspace_create - build the plane-wave sphere and FFT grid for a cell
 * (the GSpace of Sec. 4.3.2 for the wavefunction cutoff; truncation of Sec. 2.2 / 4.3.1).
 *
 *  lattice[9]     host; rows a_1, a_2, a_3 in Cartesian bohr.
 *  nk, kpts       host; nk >= 1 k-points, kpts[3*ik + d] in crystal coordinates of the
 *                 reciprocal lattice (k = sum_d kpts_d b_d, b_i . a_j = 2 pi delta_ij).
 *  ecutwfc_ha     wavefunction cutoff E_c (Ha): plane waves with |k+G|^2/2 <= E_c are kept
 *                 (inclusive, relative slack 1e-12).
 *  grid_override  host; NULL -> grid rule: n_d = floor(sqrt(8 E_c) |a_d| / 2 pi),
 *                 N_d = smallest 2,3,5-smooth integer >= 2 n_d + 1 (the dual 4 E_c density
 *                 cutoff of Sec. 2.2).  Otherwise N_d = grid_override[d], each in [2, 512]
 *                 and 2,3,5-smooth; a grid too small for the sphere is QM_ERR_ARG.
 *  out            host; receives the handle.
 * Host-only: no CUDA call is made here.  The handle's device tables are uploaded
 * (synchronously, with cudaMalloc/cudaMemcpy) to the device that is current at the first
 * compute call using the handle; later calls must run with that same device current.
 * Make that first call outside any CUDA stream capture.
 */
qm_status qm_gspace_create(const double lattice[9], int nk, const double* kpts,
                           double ecutwfc_ha, const int grid_override[3], qm_gspace* out);

/*
 * qm_gspace_query - sizes of a gspace.
 *  grid[3]   host, may be NULL: (N1, N2, N3).
 *  npw       host, may be NULL: npw[ik] for ik < nk (array of nk ints).
 *  npw_max   host, may be NULL: max over k of npw.
 *  nk        host, may be NULL: number of k-points.
 */
qm_status qm_gspace_query(qm_gspace g, int grid[3], int* npw, int* npw_max, int* nk);

/*
 * qm_gspace_indices - host copies of the sphere of k-point ik (Sec. 4.3.2 idxgrid/g_cryst).
 *  idx     host, may be NULL: npw int32 flat grid indices (increasing).
 *  miller  host, may be NULL: npw*3 int32 crystal components m of G.
 *  kpg     host, may be NULL: npw*3 doubles, Cartesian k+G (bohr^-1).
 */
qm_status qm_gspace_indices(qm_gspace g, int ik, int32_t* idx, int32_t* miller, double* kpg);

/*
 * qm_gspace_sticks - host copies of the x-stick layout of k-point ik (the pruning of Sec. 4.3.3):
 *  nstick    host, may be NULL: number of x-sticks (distinct (i2, i3) holding a plane wave).
 *  stick_yz  host, may be NULL: nstick * 2 int32, (i2, i3) of each stick in the order the FFT
 *            kernels use (increasing i2 + N2 i3).
 *  ngtile    host, may be NULL: at the Gamma point, the tiles of qm_hpsi_gamma's forward x pass
 *            (0 at other k-points).
 *  gtile     host, may be NULL: ngtile * 32 * 2 int32, per tile slot (stick index or -1 for an
 *            empty slot, slot of the stick holding -G); a stick (i2, i3) and its partner
 *            (-i2, -i3) share a tile.
 * Host-only.
 */
qm_status qm_gspace_sticks(qm_gspace g, int ik, int* nstick, int32_t* stick_yz, int* ngtile, int32_t* gtile);

/* qm_gspace_destroy - free the handle and its device tables/workspace (NULL is a no-op).
 * Synchronises the device first, so in-flight work that uses the handle completes. */
void qm_gspace_destroy(qm_gspace g);

/*
 * qm_hpsi - out = H(k) psi for a block of nb bands (Eq. KSHamMat with the KB term;
 * the local part by the IFFT / V(r) / FFT recipe of Sec. 4.3, stick-pruned as in
 * Sec. 4.3.3; kinetic 1/2|k+G|^2 in G-space as in Sec. 4.3).
 *
 *  g, ik      gspace and k-point index (0 <= ik < nk).
 *  nb         number of bands, >= 0 (0 is a no-op).
 *  psi        device, nb rows of npw(ik) complex, row stride ld_psi (>= npw).
 *             QM_FP64: double[2]; QM_MIXED: float[2].
 *  vloc_r     device, N1*N2*N3 doubles, V(r_j) in Ha on the grid, x fastest.
 *  nproj      number of projectors, >= 0.
 *  beta       device, nproj rows of npw(ik) complex (same element type as psi),
 *             row stride ld_beta (>= npw); may be NULL when nproj == 0.
 *  D          device, nproj doubles (diagonal KB coefficients, Ha).
 *  out        device, nb rows, row stride ld_out (>= npw), same element type as psi;
 *             overwritten.  Must not overlap psi.
 *  prec       QM_FP64 or QM_MIXED.
 *  stream     cudaStream_t (NULL = default stream).  Asynchronous: returns after the
 *             launches are queued.  Uses the handle's device workspace.  QM_MIXED with
 *             nproj > 0 runs the nonlocal part on a second stream owned by the handle,
 *             forked from and joined back to `stream` with events (capturable in a graph).
 * Errors: QM_ERR_ARG (sizes, NULL pointers, misaligned rows), QM_ERR_OOM (workspace),
 *         QM_ERR_CUDA (launch failure).
 */
qm_status qm_hpsi(qm_gspace g, int ik, int nb,
                  const void* psi, int ld_psi,
                  const double* vloc_r,
                  int nproj, const void* beta, int ld_beta, const double* D,
                  void* out, int ld_out,
                  qm_precision prec, void* stream);

/*
 * qm_hpsi_gamma - out = H(Gamma) psi for real wavefunctions, two bands per FFT: the same operator
 * and arguments as qm_hpsi, for the Gamma-point cells the paper runs with real wavefunctions.
 * At k = 0 a state whose real-space values are real has psi(-G) = conj(psi(G)), and H (real V,
 * projectors with beta_p(-G) = +-conj(beta_p(G))) keeps that property.  Bands 2j and 2j+1 are
 * transformed together as psi_2j + i psi_2j+1; after the multiplication by V(r) the forward
 * transform F separates as (V psi_2j)(G) = (F(G) + conj F(-G))/2 and (V psi_2j+1)(G) =
 * (F(G) - conj F(-G))/(2i), so the FFT path does half the transforms of qm_hpsi.  The nonlocal
 * part is the same as qm_hpsi's.  An odd nb pairs the last band with zero.
 *
 *  Requirements: k-point ik is Gamma (kpts == 0); every band satisfies psi(-G) = conj(psi(G))
 *  (for other states the local part of the result is not H psi).
 * Errors: as qm_hpsi, plus QM_ERR_ARG when ik is not the Gamma point.
 */
qm_status qm_hpsi_gamma(qm_gspace g, int ik, int nb,
                        const void* psi, int ld_psi,
                        const double* vloc_r,
                        int nproj, const void* beta, int ld_beta, const double* D,
                        void* out, int ld_out,
                        qm_precision prec, void* stream);

/*
 * qm_hpsi_check - synchronise `stream` and read (and clear) the handle's sticky error word:
 * QM_ERR_TIMEOUT if a bounded device-side wait of a tensor-core kernel launched by an earlier
 * qm_hpsi(QM_MIXED) or qm_precond_apply call on this handle expired since the last check (the
 * outputs of such a call are undefined), else QM_OK.  qm_davidson checks it itself.
 */
qm_status qm_hpsi_check(qm_gspace g, void* stream);

/*
 * qm_hpsi_prepare - prepare the projectors of k-point ik for the precision form: the
 * Hamiltonian's projectors are fixed for a k-point (Sec. 2.3, KB form; Sec. 5, the KSHam of a
 * k-point holds them across all its H psi calls), so their 3-term BF16 split into the two
 * tensor-core operand layouts of the nonlocal part is done once here instead of on every
 * qm_hpsi(QM_MIXED) call.
 *
 *  g, ik          gspace and k-point.
 *  nproj, beta, ld_beta   as in qm_hpsi (beta: device, FP32 complex).  nproj = 0 releases the
 *                 k-point's prepared projectors (beta may be NULL).
 *  stream         cudaStream_t; the split runs asynchronously on it.
 * A later qm_hpsi(g, ik, ..., QM_MIXED) whose nproj, beta and ld_beta are the prepared ones
 * uses the prepared operands (the result is identical: the same split of the same values).  The
 * caller must not change the contents of beta while it is prepared; call again after changing
 * it.  Device memory: 12 bytes per projector coefficient (two layouts of three BF16 planes),
 * owned by the handle (freed by this call with nproj = 0, a larger re-preparation, or
 * qm_gspace_destroy).  Not for use inside a stream capture (allocates).
 * Errors: QM_ERR_ARG, QM_ERR_OOM, QM_ERR_CUDA.
 */
qm_status qm_hpsi_prepare(qm_gspace g, int ik, int nproj, const void* beta, int ld_beta, void* stream);

/*
 * qm_hpsi_noalloc - the H psi operator of qm_hpsi for callers that cannot allocate device
 * memory.  The paper has no counterpart: this is a deployment variant of qm_hpsi.
 *
 * Who needs it: code running under an allocator that owns the whole device heap (for
 * example a host framework that reserves the free memory up front and forbids cudaMalloc
 * afterwards), and latency-critical loops where cudaMalloc/cudaFree would synchronise the
 * device or could fail for lack of free memory.  This call allocates nothing: it calls
 * no cudaMalloc, cudaFree or other allocating routine, not even on first use of a handle.
 * The caller still passes every input and output (same arguments and meaning as qm_hpsi).
 * All scratch - V(r) in the FFT layout, the projections, the split-K partial sums, the FFT
 * stick buffer and, when needed, a copy of the k-point's gspace tables - lives in one fixed
 * device array of QM_HPSI_NOALLOC_SCRATCH_BYTES inside the library; every GPU that loads
 * the library holds it until the process exits (the driver makes it resident when the
 * library's device code and data are loaded on that GPU, which with CUDA's lazy loading
 * can be the first call of this entry point).
 *
 *  - Every call looks up the array's device address (cudaGetSymbolAddress); the first call
 *    on a device may load the library's device code there, so make that first call before
 *    any CUDA stream capture.
 *  - Every call shares the one array and leaves its contents behind.  Calls whose GPU work
 *    overlaps (different streams, or different threads without ordering) race on it:
 *    issue them on one stream.  No scratch byte needs to start at zero; each call writes
 *    everything it reads.
 *  - The k-point's FFT tables: when the handle already holds them on the device (any earlier
 *    qm_hpsi, qm_hpsi_prepare or qm_davidson call with the handle uploaded them), they are
 *    read in place and the call only queues work on `stream`.  Otherwise every call copies
 *    them from the handle's host copies into the array; that source is pageable host memory,
 *    so the host waits until the stream's earlier work is done before each copy.
 *  - Numerics: QM_FP64 is the FP64 path of qm_hpsi.  QM_MIXED runs the FP32 FFT path of
 *    qm_hpsi but its nonlocal projection and application as FP32 SIMT products (qm_hpsi uses
 *    BF16x3 tensor-core products, whose operand planes would need scratch of their own); both
 *    are FP32-accurate (measured against the FP64 oracle: about 1e-7 per band on small cells).
 *  - A problem whose scratch exceeds the array is rejected with QM_ERR_ARG and a message
 *    giving the bytes it needs (tables + N1*N2*N3 reals + nproj*nb complex + one band of
 *    the stick buffer); use qm_hpsi for those.
 * Errors: as qm_hpsi, plus the size rejection above.
 */
#define QM_HPSI_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)
qm_status qm_hpsi_noalloc(qm_gspace g, int ik, int nb,
                          const void* psi, int ld_psi,
                          const double* vloc_r,
                          int nproj, const void* beta, int ld_beta, const double* D,
                          void* out, int ld_out,
                          qm_precision prec, void* stream);

/*
 * Batched H psi (the batched form: every band x k-point x cell of many independent cells of
 * uneven size in ONE persistent launch, captured in a CUDA graph).
 *
 * A batch is a plan bound to its buffers: qm_batch_create takes the jobs (each one the
 * argument list of qm_hpsi), lays the work of all of them out as one list of work items
 * (V layout, partial projections, x-stick transforms, yz-plane transforms with the V
 * multiply, projection reductions, x-stick forward transforms with the gather and kinetic
 * term, nonlocal application), allocates the intermediate buffers, and captures the launch
 * in a CUDA graph.  qm_batch_run then replays it: one kernel launch computes
 * out_j = H(k_j) psi_j for every job j, with the numerics of qm_hpsi in the same precision
 * (FFT path identical; nonlocal products accumulated in the working precision, FP32 in
 * QM_MIXED instead of the single-call tensor-core path).
 *
 * The work items are ordered in groups of jobs whose stick buffers hold about group_mb MB,
 * the phases of consecutive groups interleaved as a software pipeline, so the intermediate
 * data of a group is still in L2 when its next phase reads it.  The shape of the launch
 * (resident CTAs per SM; grid points per FFT work item, from which the lines per x-stick item
 * and the bands per yz-plane item follow; the group size; the radix order of the FFT plans) is
 * either given or picked by the autotuner, which times three replays of each candidate (after
 * one warm-up) with CUDA events on `stream`: every feasible (CTAs per SM, points per item) pair
 * at 24 MB groups and radix order 1, then the other group sizes (48 MB, one group) at the best
 * pair, then radix order 2 at the best shape; the fastest is kept.  The radix order changes the
 * rounding, not the operator: both orders give the same H psi to FFT round-off.
 */
typedef struct {
    qm_gspace g;            /* gspace of the job's cell (device tables on the current device) */
    int ik;                 /* k-point of g */
    int nb;                 /* bands, >= 1 */
    const void* psi;        /* device, as qm_hpsi */
    int ld_psi;
    int nproj;              /* >= 0 */
    const double* vloc_r;   /* device, as qm_hpsi; jobs with the same (g, vloc_r) share its layout */
    const void* beta;       /* device, as qm_hpsi (may be NULL when nproj == 0) */
    int ld_beta;
    int ld_out;
    const double* D;        /* device, as qm_hpsi */
    void* out;              /* device, as qm_hpsi; the out blocks of different jobs must not overlap */
} qm_hpsi_job;

typedef struct qm_batch_s* qm_batch;   /* opaque, library-owned */

typedef struct {
    int ctas_per_sm;   /* resident CTAs per SM, 1..8; 0 = autotune */
    int item_points;   /* target grid points per FFT work item, 256..65536; 0 = autotune */
    int group_mb;      /* stick-buffer megabytes per pipelined group of jobs, 1..4096; -1 = one
                          group (the work items of each phase of all jobs together); 0 = autotune */
    int fft_order;     /* radix order of the FFT plans: 1 = large radices first (8s, 4, 2, 9s, 3,
                          5s, the single-call order), 2 = the same radices reversed; 0 = autotune */
} qm_batch_shape;

typedef struct {
    int ctas_per_sm, item_points;  /* shape in use */
    int group_mb;                  /* group size in use (-1: one group) */
    int grid;                      /* CTAs of the persistent launch */
    int items;                     /* work items per replay */
    int cells;                     /* distinct (gspace, vloc_r) pairs */
    int candidates;                /* shapes the autotuner timed (0: shape given) */
    long long band_applies;        /* sum over jobs of nb */
    long long smem_bytes;          /* dynamic shared memory per CTA */
    long long device_bytes;        /* device memory owned by the batch */
    double tuned_ms;               /* autotuner's best median time per replay (ms; 0 if not tuned) */
    int fft_order;                 /* radix order in use: 0 = large radices first, 1 = reversed */
} qm_batch_info;

/*
 * qm_batch_create - build (and, with shape NULL or zero fields, autotune) a batch.
 *  njobs, jobs   host array of njobs >= 1 job descriptions (copied; the buffers they point
 *                to must stay valid and keep their addresses for the life of the batch).
 *  prec          QM_FP64 or QM_MIXED (element types of psi/beta/out as in qm_hpsi).
 *  shape         host, may be NULL (autotune both fields).
 *  stream        cudaStream_t used by the autotuner.  Autotuning REPLAYS THE BATCH several
 *                times: every out block is written.  Synchronous (returns when done).
 *  out           host; receives the batch.
 * Make this call outside any stream capture.  Errors: QM_ERR_ARG (a job fails qm_hpsi's
 * checks, or two out blocks overlap), QM_ERR_UNSUPPORTED (shape does not fit an SM, more
 * than 1024 projectors in a job), QM_ERR_OOM, QM_ERR_CUDA, QM_ERR_TIMEOUT (while tuning).
 */
qm_status qm_batch_create(int njobs, const qm_hpsi_job* jobs, qm_precision prec,
                          const qm_batch_shape* shape, void* stream, qm_batch* out);

/* qm_batch_run - replay the batch's graph on `stream` (asynchronous; one kernel launch and
 * one memset).  Replays of one batch must be serialised (they share its buffers). */
qm_status qm_batch_run(qm_batch b, void* stream);

/* qm_batch_check - synchronise `stream` and read the batch's device error word:
 * QM_ERR_TIMEOUT if a bounded device-side wait of the last replay expired, else QM_OK. */
qm_status qm_batch_check(qm_batch b, void* stream);

/* qm_batch_hold - failure-detection test hook of the bounded waits (not part of the method).
 * job >= 0: from the next replay on, the last-phase work items of that job wait for one more
 * completion than will ever arrive, so their bounded waits expire, the launch gives up and
 * qm_batch_check reports QM_ERR_TIMEOUT (the outputs of that replay are undefined); job = -1
 * restores normal replays.  spin_limit: polls per bounded wait (0 = the library default of
 * 2^24); a small value makes the expiry quick.  Synchronises the device.  Errors: QM_ERR_ARG,
 * QM_ERR_CUDA. */
qm_status qm_batch_hold(qm_batch b, int job, long long spin_limit);

/* qm_batch_query - shape, sizes and tuning result of a batch. */
qm_status qm_batch_query(qm_batch b, qm_batch_info* info);

/* qm_batch_destroy - synchronise the device and free the batch (NULL is a no-op). */
void qm_batch_destroy(qm_batch b);

/* Options of qm_davidson (zero-initialise, then set what you need; 0 / 0.0 = default). */
typedef struct {
    double tol;          /* convergence: max_n ||H x_n - eps_n x_n||_2 <= tol (Ha), ||x_n||_2 = 1;
                            default 1e-8 */
    int max_iter;        /* maximum Rayleigh-Ritz steps; default 100 */
    int nvecx;           /* maximum basis size, >= 2 nb (clamped to npw); default 4 nb */
    qm_precision prec;   /* QM_FP64: every step in FP64.  QM_MIXED: H psi in FP32 (qm_hpsi
                            QM_MIXED) and the subspace products as BF16x3 tensor-core products
                            (FP32 accuracy, see mixed_ortho) until the largest residual falls
                            below mixed_switch; then the Ritz vectors are re-orthonormalised and
                            H applied to them in FP64, and the iterations continue with FP64
                            H psi to tol.  In that FP64 phase, when nconv < nb, the basis is
                            anchored on the exact Ritz vectors of each restart: products that
                            only involve small quantities (couplings through the anchors'
                            residuals, later directions, small Ritz coefficients) stay on the
                            tensor cores, the rest is FP64, and restarts, convergence and exit
                            recompute the Ritz vectors in FP64; an anchored phase whose best
                            residual stops halving for 12 steps (or lasts 60) continues in plain
                            FP64.  Eigensolves, residual norms and band energies are FP64 in
                            every form. */
    int precond;         /* 0 = Teter-Payne-Allan diagonal preconditioner; 1 = learned (the network
                            `mlp`), with TPA taking over for the rest of the call if the largest
                            residual fails to fall below precond_stall x its value 4 steps earlier */
    double mixed_switch; /* QM_MIXED: residual (Ha) where FP64 takes over (or earlier if the
                            residual, once below 1e-3, stops halving over 10 steps); 0 -> 1e-4 */
    int nconv;           /* only the lowest nconv bands must reach tol (1..nb; 0 -> nb); the
                            other nb - nconv trial vectors are a buffer that speeds convergence */
    int mixed_ortho;     /* QM_MIXED, FP32 phase: 0 (default) = every subspace product on the
                            tensor cores (BF16x3 split, FP32 accumulation, basis orthonormal to
                            about 1e-7); 1 = the second Gram-Schmidt pass's coefficients and the
                            second Cholesky-QR pass in FP64 (basis orthonormal to FP64 round-off) */
    double* history;     /* host, may be NULL: max_iter doubles, the largest residual among the
                            nconv bands after each Rayleigh-Ritz step */
    const float* mlp;    /* precond = 1: device, QM_MLP_NPARAM floats (see qm_mlp_forward) */
    double precond_stall; /* precond = 1: stall ratio of the fallback rule; 0 -> 0.8, >= 1: never
                             fall back */
    int plain_restart;   /* 0 (default) = thick restart: when the basis is full it restarts from the
                            Ritz vectors AND the new directions of the previous step's Ritz vectors
                            of the unconverged bands (GD+k: Stathopoulos & Saad, ETNA 7, 163 (1998)),
                            as many as fit beside the next corrections; 1 = plain restart from the
                            Ritz vectors only */
    int fp64_exact;      /* QM_MIXED, FP64 phase: 0 (default) = its plane-wave-length products (H_sub
                            columns, Ritz vectors, orthogonalisation passes, and the nonlocal
                            GEMMs of its H psi) in double-FP32 arithmetic: FP64 operands split into
                            two FP32 halves, products and sums by error-free transformations on the
                            FP32 pipe, partial sums in FP64 (about 2^-46 relative accuracy, 47-bit
                            rather than 53-bit); 1 = those products in FP64 arithmetic.  QM_FP64
                            is FP64 arithmetic throughout, whatever this field says */
} qm_davidson_opts;

/* Counters of one qm_davidson call (the paper's "H-psi calls" are band_applies / nb). */
typedef struct {
    int iterations;          /* Rayleigh-Ritz steps taken */
    int converged;           /* 1 if the nconv lowest residual norms reached tol */
    long long band_applies;  /* number of single-band H psi applications */
    double max_residual;     /* max over the nconv bands of ||H x_n - eps_n x_n||_2 at exit (Ha) */
    double seconds;          /* host wall time of the call */
    int iterations_mixed;    /* QM_MIXED: Rayleigh-Ritz steps taken in the FP32 phase */
    long long band_applies_mixed;  /* QM_MIXED: H psi applications done in FP32 */
    int precond_fallback;    /* precond = 1: Rayleigh-Ritz step after which TPA replaced the
                                network (0: the network was used throughout) */
    int restarts;            /* basis restarts */
    long long restart_kept;  /* previous-step directions kept over all thick restarts */
} qm_davidson_stats;

/*
 * qm_davidson - lowest nb eigenpairs of H(k) by block Davidson (Sec. 5, dft module:
 * matrix-free Davidson that only applies H to blocks of trial vectors; Eq. KSHamMat
 * with the KB term is the operator, applied as in qm_hpsi).
 *
 *  g, ik, nb      gspace, k-point, number of bands (1 <= nb <= npw/2).
 *  psi_inout      device, nb rows of npw(ik) complex double, row stride ld_psi >= npw.
 *                 In: starting block (any linearly independent vectors; orthonormalised
 *                 internally).  Out: orthonormal Ritz vectors, ordered like eig_out.
 *  vloc_r, nproj, beta, ld_beta, D   as in qm_hpsi (FP64 element types).
 *  opts           host, may be NULL (defaults).
 *  eig_out        host, nb doubles: Ritz values in increasing order (Ha).
 *  stats          host, may be NULL.
 *  stream         cudaStream_t.  Synchronous with respect to the host: the call returns
 *                 after the last iteration; it reads small results (Ritz values, residual
 *                 norms) back every iteration.
 * Uses a grow-only device workspace owned by the handle (about (2 nvecx + 5 nb) npw
 * complex doubles plus O(nvecx^2)).
 * Errors: QM_ERR_ARG, QM_ERR_OOM, QM_ERR_CUDA; QM_ERR_NUMERIC (non-finite values,
 * rank-deficient start); QM_ERR_NOT_CONVERGED (max_iter reached: outputs hold the last
 * Ritz pairs).
 */
qm_status qm_davidson(qm_gspace g, int ik, int nb, void* psi_inout, int ld_psi,
                      const double* vloc_r, int nproj, const void* beta, int ld_beta,
                      const double* D, const qm_davidson_opts* opts, double* eig_out,
                      qm_davidson_stats* stats, void* stream);

/* One problem of qm_davidson_batched: the arguments of qm_davidson. */
typedef struct {
    qm_gspace g;
    int ik;
    int nb;
    void* psi_inout;            /* device, as qm_davidson */
    int ld_psi;
    int nproj;
    const double* vloc_r;       /* device */
    const void* beta;           /* device */
    int ld_beta;
    const double* D;            /* device */
    double* eig_out;            /* host, nb doubles */
    qm_davidson_stats* stats;   /* host, may be NULL */
    double* history;            /* host, may be NULL: max_iter doubles (replaces opts->history) */
    qm_status status;           /* out: this job's status */
} qm_davidson_job;

/*
 * qm_davidson_batched - many independent Davidson problems (the k-points of a cell, or
 * cells) solved concurrently (the batched form applied to the eigensolver).  Worker host
 * threads (max_concurrent, 0 = one per job) take the jobs in order; each runs qm_davidson on
 * its own CUDA stream with its own device workspace (the job's gspace tables are shared, not
 * copied), so the jobs' latency-bound steps and host synchronisations overlap on the GPU.
 * The results are those of qm_davidson for each job (the same options `opts`, except the
 * per-job `history`).  The workers' streams start after the work queued on `stream` and
 * `stream` is ordered after them; the call returns when every job is done.
 * Returns QM_OK, the first error of a job other than QM_ERR_NOT_CONVERGED, or
 * QM_ERR_NOT_CONVERGED if some job did not converge; each job's own status is in
 * jobs[i].status.  Jobs may share a gspace and a k-point only if their buffers differ.
 */
qm_status qm_davidson_batched(int njobs, qm_davidson_job* jobs, const qm_davidson_opts* opts,
                              int max_concurrent, void* stream);

/*
 * qm_precond_apply - the residual and correction steps of one Davidson iteration on their
 * own (Sec. 5, dft module: the correction step of the matrix-free Davidson; the diagonal
 * Teter-Payne-Allan preconditioner, Phys. Rev. B 40, 12255 (1989), or the learned network),
 * with the kernels qm_davidson launches for them:
 *   r_n      = HX_n - eps_n X_n,            rnorm2_n = ||r_n||^2,
 *   T_n      = sum_G T_G |X_n(G)|^2 / sum_G |X_n(G)|^2,   T_G = |k+G|^2 / 2,
 *   delta_n  = K_n(G) r_n(G),  K = K_TPA(T_G / T_n) (precond 0) or the network of
 *              qm_mlp_forward on the features (T_G/T_n, eps_n/T_n, (H_GG - eps_n)/T_n)
 *              (precond 1; H_GG from qm_hamiltonian_diag).
 *
 *  g, ik      gspace and k-point.
 *  n          number of bands, 0 <= n <= 65535 (0 is a no-op).
 *  X, HX      device, n rows of npw(ik) complex double, row stride ld (>= npw): Ritz vectors
 *             (any non-zero rows; T_n is normalised by the row's own norm) and H applied to them.
 *  eps        device, n doubles: the Ritz values eps_n.
 *  precond    0 = TPA, 1 = learned (mlp: device, QM_MLP_NPARAM floats, as qm_mlp_forward;
 *             hdiag: device, npw doubles, the diagonal of H(k); both may be NULL for TPA).
 *  R, delta   device, n rows, row stride ld: outputs r_n and delta_n (must not overlap the inputs
 *             or each other).
 *  rnorm2     device, n doubles: output ||r_n||^2 (FP64).
 *  tkin       device, n doubles: output T_n (FP64).
 *  stream     cudaStream_t.  precond 0 is asynchronous; precond 1 synchronises the stream to
 *             read the network's error word (the handle's workspace holds it: same one-stream
 *             rule as qm_hpsi).
 * Arithmetic: FP64 (TPA); the network in BF16 with FP32 accumulation, K applied in FP64.
 * Errors: QM_ERR_ARG, QM_ERR_CUDA, QM_ERR_OOM, QM_ERR_TIMEOUT (a bounded wait of the network).
 */
qm_status qm_precond_apply(qm_gspace g, int ik, int n, const void* X, const void* HX, int ld, const double* eps,
                           int precond, const float* mlp, const double* hdiag, void* R, void* delta, double* rnorm2,
                           double* tkin, void* stream);

/*
 * qm_hamiltonian_diag - the diagonal of H(k) in the plane-wave basis (Eq. KSHamMat with the KB
 * term of Sec. 2.3):  hdiag[G] = |k+G|^2/2 + Vt(0) + sum_p D_p |beta_p(G)|^2, Vt(0) = the mean
 * of V(r) over the grid.  The learned preconditioner's third feature is (hdiag - eps_n) / T_n.
 *  vloc_r, nproj, beta, ld_beta, D   as in qm_hpsi, FP64 (beta may be NULL when nproj == 0).
 *  hdiag      device, npw(ik) doubles (output).
 * FP64, asynchronous on stream (partial sums of V in the handle's workspace: same one-stream
 * rule as qm_hpsi).  Errors: QM_ERR_ARG, QM_ERR_OOM, QM_ERR_CUDA.
 */
qm_status qm_hamiltonian_diag(qm_gspace g, int ik, const double* vloc_r, int nproj, const void* beta, int ld_beta,
                              const double* D, double* hdiag, void* stream);

/*
 * qm_eigh_lowest - lowest nev eigenpairs of a complex Hermitian m x m matrix in FP64: the
 * dense eigensolver of the Davidson Rayleigh-Ritz step, exposed on its own.  Householder
 * reduction to real tridiagonal form, multisection on Sturm counts for the wanted
 * eigenvalues, inverse iteration (orthogonalised within clusters closer than 1e-5 |T|),
 * back-transformation (Golub & Van Loan, Matrix Computations, Ch. 8).
 *
 *  A       device, m x m complex double (row-major, ld lda >= m); only read (the Hermitian
 *          part (A + A^H)/2 is what is diagonalised).
 *  evals   device, nev doubles, increasing.
 *  Y       device, m x nev complex double, row-major with ld ldy >= nev: column j is the
 *          unit eigenvector of evals[j].
 *  stream  cudaStream_t.  Allocates its workspace with cudaMallocAsync on the stream.
 * 1 <= nev <= m <= 6400.  Errors: QM_ERR_ARG, QM_ERR_UNSUPPORTED, QM_ERR_CUDA, QM_ERR_OOM.
 */
qm_status qm_eigh_lowest(int m, int nev, const void* A, int lda, double* evals, void* Y, int ldy,
                         void* stream);

/*
 * qm_zgemm - the plane-wave-length complex products of the Davidson step (the Gram-Schmidt
 * and H_sub products, Sec. 5 dft module) and of the nonlocal term (Sec. 2.3), exposed on their
 * own so that their arithmetic can be checked:
 *   op 0 (cn): C[m][n] = sum_k conj(A[m][k]) B[n][k]     A: M x K, B: N x K (k contiguous)
 *   op 1 (tn): C[m][n] = sum_k A[k][m] B[k][n]           A: K x M, B: K x N (m, n contiguous)
 *  arith   0 = FP64 arithmetic; 1 = double-FP32 (the precision form's FP64 phase, see
 *          qm_davidson_opts.fp64_exact): operands split into two FP32 halves, error-free
 *          products and sums on the FP32 pipe, per-tile sums in FP64; 2 = 3-term BF16 split
 *          products on the tensor cores accumulated in FP32 (the precision form's FP32 phase;
 *          FP32-level accuracy; synchronises the stream).
 *  A, B, C device, complex double, row-major with the leading dimensions given; C is written.
 *  stream  cudaStream_t.  Split-K partial sums and tensor-core workspaces are allocated with
 *          cudaMallocAsync on the stream.
 * M, N, K >= 1.  Errors: QM_ERR_ARG, QM_ERR_CUDA, QM_ERR_OOM, QM_ERR_TIMEOUT (arith 2).
 */
qm_status qm_zgemm(int op, int arith, int M, int N, int K, const void* A, int lda, const void* B, int ldb, void* C,
                   int ldc, void* stream);

/*
 * qm_tddft_taylor - real-time propagation by the truncated Taylor series of the propagator
 * (Sec. 5, "tddft" module, expoper submodule):
 *     psi <- sum_{r=0}^{order} (-i dt)^r / r!  H^r psi
 * with H the operator of qm_hpsi (same g, ik, vloc_r, nproj, beta, ld_beta, D, prec).  The terms
 * are built as u_r = (-i dt / r) H u_{r-1}, u_0 = psi: one qm_hpsi per term, then one element-wise
 * kernel that scales u_r in place and adds it to psi.
 *
 *  psi     device, in/out, nb rows of npw(ik) complex (double[2] for QM_FP64, float[2] for
 *          QM_MIXED), row stride ld_psi >= npw.
 *  dt      time step in atomic units of time (hbar / Ha), finite; order in [0, 64] (order 0 or
 *          nb 0: nothing is done).
 *  work    device, caller-owned scratch of 2 * nb * ld_psi complex elements of psi's type; must
 *          not overlap psi; its contents on return are the last two terms.
 *  stream  cudaStream_t; asynchronous.  Uses the handle's workspace like qm_hpsi (so the same
 *          one-stream-per-handle rule applies); with QM_MIXED the projectors prepared by
 *          qm_hpsi_prepare for this beta are used.
 * Errors: QM_ERR_ARG (sizes, NULL pointers, order or dt out of range, work overlapping psi;
 *         nothing launched), QM_ERR_OOM, QM_ERR_CUDA.
 */
qm_status qm_tddft_taylor(qm_gspace g, int ik, int nb, void* psi, int ld_psi, const double* vloc_r,
                          int nproj, const void* beta, int ld_beta, const double* D,
                          double dt, int order, void* work, qm_precision prec, void* stream);

/*
 * qm_tddft_etrs - one enforced-time-reversal-symmetry step (Sec. 5, "tddft" module, prop
 * submodule): psi <- U(dt/2; H_next) U(dt/2; H_now) psi, each U the Taylor series of
 * qm_tddft_taylor of the given order.  H_now and H_next are the operator of qm_hpsi with the local
 * potentials vloc_now and vloc_next (device, N_r doubles each); the projectors and D are shared.
 * The Hamiltonian of this library has no density functional, so the potential at the end of the
 * step (the H[psibar] of a self-consistent propagation) is supplied by the caller.  Other
 * arguments, errors and asynchrony as qm_tddft_taylor.
 */
qm_status qm_tddft_etrs(qm_gspace g, int ik, int nb, void* psi, int ld_psi, const double* vloc_now,
                        const double* vloc_next, int nproj, const void* beta, int ld_beta, const double* D,
                        double dt, int order, void* work, qm_precision prec, void* stream);

/*
 * qm_gw_mel - plane-wave matrix elements of the GW module (Sec. 5, "gw" module, matrix_elements):
 *     M_nn'(G) = <n k+q| exp(i(q+G).r) |n' k> = sum_{G2} conj(c_{n,k+q}(G + G2)) c_{n',k}(G2)
 * for G on the sphere |q+G|^2/2 <= E_eps, by the paper's route: both sets of states to real space
 * with the stick-pruned inverse FFT of qm_hpsi, the product conj(u_n(r)) u_n'(r) of every pair,
 * one forward FFT per pair gathered onto the sphere of q.
 *
 *  g, ik_left, ik_right  wavefunction gspace and the k-points k+q (left states) and k (right).
 *  nl, psi_l, ld_l       device, nl rows on the sphere of ik_left (ld_l >= its npw).
 *  nr, psi_r, ld_r       device, nr rows on the sphere of ik_right.
 *  geps, iq              gspace of the E_eps sphere: the same FFT grid as g, and its k-point iq
 *                        equal to kpts[ik_left] - kpts[ik_right] (crystal coordinates, 1e-10).
 *  M, ld_m               device, nl * nr rows (row n * nr + n') of npw(geps, iq) complex, ld_m >=
 *                        that npw; overwritten.
 *  prec                  QM_FP64 (double[2] everywhere) or QM_MIXED (float[2]: FP32 transforms).
 *  stream                asynchronous on the stream; uses g's workspace (two full FFT boxes per
 *                        state, N1 N2 N3 complex each, plus stick buffers of at most 256 MB each).
 * The result is exact (to rounding) when the grid holds every G + G2 without wrap-around, as the
 * grid rule's density grid does for E_eps <= the wavefunction cutoff.
 * Errors: QM_ERR_ARG (sizes, NULL pointers, grids or q that do not match), QM_ERR_OOM, QM_ERR_CUDA.
 */
qm_status qm_gw_mel(qm_gspace g, int ik_left, int ik_right, int nl, const void* psi_l, int ld_l, int nr,
                    const void* psi_r, int ld_r, qm_gspace geps, int iq, void* M, int ld_m,
                    qm_precision prec, void* stream);

/*
 * qm_scf - Kohn-Sham self-consistency around qm_davidson (Sec. 2.1: n -> V -> {psi} -> n_out ->
 * mix, until n_out = n; Sec. 5, dft module scf with density mixing).
 *   V(r) = V_ext(r) + V_H[n](r) + v_xc(n(r)):  V_H(G) = 4 pi n(G) / |G|^2 on the density sphere
 *          |G|^2/2 <= 4 E_c (G = 0 left out: neutralising background); v_xc the local density
 *          approximation (Slater exchange + Perdew-Zunger correlation, unpolarised; no
 *          exchange-correlation where n <= 1e-12).
 *   n(r)  = sum_k w_k sum_{n < nelec/2} 2 |psi_nk(r)|^2 (insulating occupations, spin-degenerate).
 *   mixing: Anderson (equal-weight modified Broyden) on the density residual F = n_out - n_in with
 *          the last `history` differences and factor alpha, from the uniform density nelec / Omega.
 *   converged when (Omega / N_r) sum_r |n_out - n_in| <= tol (electrons).
 *
 *  g          wavefunction gspace (all its k-points take part); the grid must hold the density
 *             sphere (the grid rule's grid does), else QM_ERR_ARG.
 *  nelec      electrons, even, >= 2; nb >= nelec/2 bands are solved per k-point.
 *  wk         host, nk weights summing to 1.
 *  psi        host array of nk device pointers: nb rows of complex double (ld_psi >= npw); the
 *             starting states in, the last Ritz vectors out.
 *  vion_r     device, N_r doubles: V_ext on the grid (x fastest).
 *  nproj, beta, ld_beta, D   projectors: beta is a host array of nk device pointers (or NULL when
 *             nproj == 0), each as qm_hpsi's; D device.
 *  opts       host, may be NULL (defaults below).
 *  eigs       host, nk * nb doubles: the last Ritz values.
 *  rho_r, vloc_r   device, N_r doubles each: the last input density and its potential.
 *  stats      host, may be NULL.
 *  stream     cudaStream_t; synchronous with respect to the host.  Allocates its densities and
 *             transform buffers with cudaMalloc for the call; qm_davidson uses g's workspaces.
 * Errors: QM_ERR_ARG, QM_ERR_OOM, QM_ERR_CUDA, QM_ERR_NUMERIC; QM_ERR_NOT_CONVERGED (max_iter
 *         reached: the outputs hold the last step).
 */
typedef struct {
    double tol;        /* density residual (electrons); default 1e-8 */
    int max_iter;      /* self-consistency steps; default 50 */
    double alpha;      /* mixing factor in (0, 1]; default 0.5 */
    int history;       /* differences kept by the mixing, 0..8 (0: linear mixing); default 4 */
    double dav_tol;    /* qm_davidson residual tolerance (Ha) of every step; default 1e-9 */
    int dav_max_iter;  /* qm_davidson max_iter; default 100 */
    qm_precision prec; /* qm_davidson form; default QM_FP64 */
} qm_scf_opts;

typedef struct {
    int iterations;          /* self-consistency steps taken */
    int converged;           /* 1 if the density residual reached tol */
    double drho;             /* last density residual (electrons) */
    long long band_applies;  /* H psi band applications of all the Davidson calls */
    double seconds;          /* host wall time of the call */
} qm_scf_stats;

qm_status qm_scf(qm_gspace g, int nelec, const double* wk, int nb, void* const* psi, int ld_psi,
                 const double* vion_r, int nproj, const void* const* beta, int ld_beta, const double* D,
                 const qm_scf_opts* opts, double* eigs, double* rho_r, double* vloc_r,
                 qm_scf_stats* stats, void* stream);

/*
 * Learned preconditioner (the learned form): a network K(f) > 0 on per-plane-wave features
 * replaces the Teter-Payne-Allan factor in the Davidson correction, delta_n(G) = K(f_nG) r_n(G).
 *
 * Network: z1 = W1 f + b1, h1 = silu(z1), z2 = W2 h1 + b2, h2 = silu(z2), z3 = w3 . h2 + b3,
 * K = K_TPA(x) softplus(z3) / log 2, silu(z) = z / (1 + e^-z): a positive factor on the TPA
 * curve K_TPA(x) = (27+18x+12x^2+8x^3)/(27+18x+12x^2+8x^3+16x^4); z3 = 0 gives TPA exactly.  Parameters: one device array of QM_MLP_NPARAM
 * floats, W1 (64 x 3, row-major W1[j][k]) | b1 (64) | W2 (64 x 64, W2[j][i], j output) | b2 (64)
 * | w3 (64) | b3 (1).  Arithmetic: BF16 weights, features and hidden activations, FP32
 * accumulation (the 64 x 64 layer of inference on the tensor cores, tcgen05).
 * Features of plane wave G of band n (scale-free): x = T_G / T_n with T_G = |k+G|^2/2 and T_n
 * the band's kinetic energy per unit norm; e = eps_n / T_n (Ritz value); d = (H_GG - eps_n) / T_n
 * with H_GG the diagonal of H(k) (qm_hamiltonian_diag).  None depends on the residual, so the
 * correction K r_n is linear in r_n.
 * Training target: the exact correction delta*_n = P_c psi_n / (psi_n^H P_c psi_n) - psi_n,
 * P_c the projector on the exact eigenspace of eigenvalue n (with its degenerate partners); loss: the mean over bands of
 * 1 - cos^2 between K.r_n and delta*_n (only the direction matters to Davidson), weighted by
 * W_n: sum_n W_n (1 - cos^2_n) / sum_n W_n.  A sample is (features, |r_G|^2, c_G =
 * Re(conj(r_G) delta*_G)); a band adds D_n = ||delta*_n||^2 (D_n = 0 excludes it) and its weight
 * W_n.  Samples are grouped by band: band b owns samples band_off[b] .. band_off[b+1]-1.
 */
#define QM_MLP_NPARAM 4481

/* qm_mlp_forward - K for n feature rows (device feats[3n], theta; K out, n floats).
 * Synchronous.  Errors: QM_ERR_ARG, QM_ERR_CUDA, QM_ERR_TIMEOUT. */
qm_status qm_mlp_forward(long long n, const float* feats, const float* theta, float* K, void* stream);

/* qm_mlp_pairs - training samples of n Ritz pairs of k-point ik from exact eigenpairs.
 *  psi, hpsi   device, n rows (ld_psi, ld_hpsi >= npw) complex double: Ritz vectors and H psi.
 *  eps         device, n Ritz values.
 *  hdiag       device, npw doubles: the diagonal of H(k) (qm_hamiltonian_diag).
 *  U, lam      device: nu exact unit eigenvectors (rows, ld_u >= npw) and eigenvalues, ascending.
 *  cluster_tol band n (the n-th lowest Ritz pair) targets eigenvalue n and its partners within
 *              cluster_tol; a band whose cluster reaches lam[nu-1] (or n >= nu) gets D = 0.
 *  feats       device, n*npw*3 floats; r2, c: n*npw floats; D, W: n floats (band-major samples).
 *              W_n = ||r_n||^2 / sum_m ||r_m||^2 over the call's bands with D_m > 0 (0 where
 *              D_n = 0): Davidson stops on its largest residual, so the bands that carry it weigh most.
 * Synchronous (allocates temporaries with cudaMallocAsync). */
qm_status qm_mlp_pairs(qm_gspace g, int ik, int n, const void* psi, int ld_psi, const void* hpsi, int ld_hpsi,
                       const double* eps, const double* hdiag, int nu, const void* U, int ld_u, const double* lam,
                       double cluster_tol, float* feats, float* r2, float* c, float* D, float* W, void* stream);

/* qm_mlp_loss_grad - loss (host double) and its gradient (device, QM_MLP_NPARAM floats) over
 * the samples; band_off: device, nband + 1 long longs; W: device, nband floats or NULL (all 1).
 * Synchronous. */
qm_status qm_mlp_loss_grad(int nband, const long long* band_off, const float* feats, const float* r2,
                           const float* c, const float* D, const float* W, const float* theta, double* loss,
                           float* grad, void* stream);

/* qm_mlp_train - `steps` full-batch Adam steps (beta1 0.9, beta2 0.999, eps 1e-8, step size
 * lr) on theta (device, updated in place) with the BF16 forward and backward kernels;
 * loss_history (host, may be NULL) receives steps + 1 losses (before each step and at the end).
 * Synchronous. */
qm_status qm_mlp_train(int nband, const long long* band_off, const float* feats, const float* r2,
                       const float* c, const float* D, const float* W, float* theta, int steps, double lr,
                       double* loss_history, void* stream);

/*
 * Instrumentation (not part of the paper's method; used by benchmarks).
 *  qm_launch_count  number of CUDA kernels this library has launched in this process.
 *  qm_prof_enable   on != 0: from now on record a pair of CUDA events on the launch stream
 *                   around every kernel launch; resets the accumulated times (any value).
 *  qm_prof_read     waits for the recorded events and returns, for kernel family
 *                   `family` (0 <= family < 18), the summed device time in ms and the number
 *                   of launches timed since the last qm_prof_enable.
 *  qm_prof_name     name of a kernel family ("" when out of range).
 */
unsigned long long qm_launch_count(void);
qm_status qm_prof_enable(int on);
qm_status qm_prof_read(int family, double* ms_total, long long* launches);
const char* qm_prof_name(int family);

/* qm_last_error - message of the last failed call on this thread ("" if none). */
const char* qm_last_error(void);

/* qm_version - library version string. */
const char* qm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QM_H */
