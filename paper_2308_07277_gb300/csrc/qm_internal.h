// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/qm.h"

namespace qm {

constexpr int kMaxStages = 12;

// Mixed-radix plan of one FFT axis.  Stage s (0-based, DIF order) works on blocks of
// length L[s] with radix r[s]; M = L[s]/r[s] butterflies per block.
struct AxisPlan {
    int n;
    int nst;
    int r[kMaxStages];
    int L[kMaxStages];
};

// sticks per tile of the Gamma-point x-forward pass (pairs in slots j and j + kGammaTile / 2)
constexpr int kGammaTile = 32;

// Per-k-point tables (device pointers unless noted).
struct KTables {
    int npw = 0;
    int nstick = 0;      // active x-sticks: distinct (i2, i3) holding >= 1 plane wave
    int nstick_pad = 0;  // row stride of the stick buffers
    int nrow = 0;        // active plane rows: distinct i3 among the sticks
    int* stick_g0 = nullptr;     // [nstick+1] first plane wave of each stick
    int* stick_plane = nullptr;  // [nstick]  i3 * ldy + i2 (position in a yz plane)
    int* rows = nullptr;         // [nrow]    active i3 values
    int2* g_code = nullptr;      // [npw]     {stick id, i1}
    double* kin = nullptr;       // [npw]     |k+G|^2 / 2
    float* kin_f = nullptr;      // [npw]     same, FP32
    // Gamma point only (k = 0): tiles of the x-forward pass of the real-wavefunction form, each
    // of kGammaTile slots {stick id (-1: empty), slot of the stick holding -G}; a stick and its
    // partner (-i2, -i3) sit in one tile, so that both G and -G are in the tile's shared memory
    bool gamma = false;
    int ngtile = 0;
    int2* gtile = nullptr;       // [ngtile * kGammaTile]
    // host copies (the device tables are uploaded from these on first use)
    std::vector<int32_t> h_idx, h_miller;
    std::vector<double> h_kpg, h_kin;
    std::vector<int> h_g0, h_plane, h_rows;
    std::vector<int2> h_code, h_gtile;
};

struct Workspace {
    void* ptr = nullptr;
    size_t bytes = 0;
};

// Projectors of one k-point prepared for the precision form's tensor-core nonlocal part
// (qm_hpsi_prepare): the BF16 planes of beta in both GEMM layouts, for calls that pass the same
// (beta, ld, nproj).
struct NlPrep {
    const void* beta = nullptr;
    int ld = 0, nproj = 0;
    void* dev = nullptr;
    size_t bytes = 0;
};

}  // namespace qm

struct qm_gspace_s {
    int device = 0;
    bool uploaded = false;   // device tables present (on `device`)
    int n[3] = {0, 0, 0};
    int ldx = 0;   // padded line length of x sticks in shared memory
    int ldy = 0;   // padded row length of a yz plane in shared memory
    double lattice[9];
    double recip[9];
    double ecut = 0;
    int nk = 0;
    std::vector<double> kpts;
    std::vector<qm::KTables> k;
    qm::AxisPlan plan[3];
    // twiddles exp(+2 pi i t / N_d), t < N_d, and the digit-reversal tables rev[p] =
    // natural index held at position p after the in-place DIF pass.
    double2* tw64[3] = {nullptr, nullptr, nullptr};
    float2* tw32[3] = {nullptr, nullptr, nullptr};
    int* rev[3] = {nullptr, nullptr, nullptr};
    std::vector<double2> h_tw[3];
    std::vector<int> h_rev[3];
    std::vector<qm::NlPrep> prep;  // per k-point prepared projectors (qm_hpsi_prepare)
    qm::Workspace ws;    // qm_hpsi workspace
    qm::Workspace dws;   // qm_davidson workspace
    // second stream of qm_hpsi(QM_MIXED): the tensor-core nonlocal part runs on it while the
    // FFT path runs on the caller's stream (fork / join events); created with the tables
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // a clone shares the device tables of its origin (owned there) and has its own
    // workspaces, stream and events, so calls on the two can run concurrently
    bool shared_tables = false;
};

namespace qm {

// error reporting (thread-local message)
qm_status fail(qm_status st, const std::string& msg);
qm_status cuda_check(cudaError_t e, const char* what);
void clear_error();

// upload the handle's tables to the current device on first use (synchronous)
qm_status ensure_device(qm_gspace g);
// a handle that shares g's uploaded device tables but owns its workspaces, stream and events
// (free with qm_gspace_destroy; destroy it before g)
qm_status gspace_clone(qm_gspace g, qm_gspace* out);

// grow-only workspace owned by a gspace handle; synchronises `stream` before regrowing.  The
// first kWsHeader bytes of the qm_hpsi workspace hold the handle's sticky error word (an int
// set by a tensor-core kernel whose bounded wait expired; read and cleared by qm_hpsi_check).
constexpr size_t kWsHeader = 256;
qm_status ensure_workspace(qm_gspace g, size_t bytes, cudaStream_t stream);
qm_status ensure_dav_workspace(qm_gspace g, size_t bytes, cudaStream_t stream);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// multiprocessor count of the current device (queried once per device)
int device_sms();
// grid for a grid-stride loop over n elements: enough CTAs of `per` threads, at most `waves`
// CTAs per multiprocessor
inline int grid_stride_blocks(size_t n, int per, int waves) {
    const size_t want = (n + per - 1) / per;
    const size_t cap = (size_t)device_sms() * waves;
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

// Allow `kernel` the device's per-CTA opt-in maximum of dynamic shared memory (minus its
// static shared memory), once per (kernel, device), and check `need` against it.  The
// attribute is global per function: setting it to each launch's own size would race between
// host threads launching the same kernel with different sizes.
qm_status allow_dynamic_smem(const void* kernel, size_t need, const char* what);

// ---- launch counting / per-kernel timing (prof.cpp) ----
enum ProfFamily { PF_VT = 0, PF_STICK_INV, PF_PLANE, PF_STICK_FWD, PF_GEMM_CN, PF_REDUCE, PF_GEMM_TN, PF_OTHER, PF_CHOL,
                  PF_TRIDIAG, PF_MULTISECT, PF_INVITER, PF_BACKTR, PF_CONVERT, PF_UMMA, PF_SPLIT, PF_BATCH, PF_MLP,
                  kProfFamilies };
void count_launch(int n);
// Counts one launch; when timing is enabled records CUDA events on `s` around the scope.
class ProfScope {
  public:
    ProfScope(int family, cudaStream_t s);
    ~ProfScope();
    ProfScope(const ProfScope&) = delete;
    ProfScope& operator=(const ProfScope&) = delete;

  private:
    int family_;
    cudaStream_t s_;
    cudaEvent_t a_ = nullptr, b_ = nullptr;
    bool active_ = false;
};

// Mixed-radix plan of an FFT length and the digit-reversal table of its in-place DIF passes:
// rev[position] = natural index.  order 0 = the radix sequence of the single-call kernels,
// order 1 = the same radices reversed (an alternative for the batched form's autotuner).
void fft_plan(int n, int order, AxisPlan& p, std::vector<int>& rev);

// ---- self-consistency loop (FFT-path parts in fft_f64.cu) ----
// work bytes for the two calls below; n_nat += the density (weight w per |u(r)|^2) of the first
// nocc rows of psi (k-point ik of g); v_nat = vion + V_H[n] + v_xc(n) with grho the density sphere
size_t scf_work_size(qm_gspace g, qm_gspace grho, int nocc);
qm_status scf_density_run(qm_gspace g, int ik, int nocc, const double2* psi, int ld, double w, double* n_nat,
                          void* work, cudaStream_t s);
qm_status scf_potential_run(qm_gspace g, qm_gspace grho, const double* n_nat, const double* vion, double* v_nat,
                            void* work, size_t work_bytes, cudaStream_t s);

// ---- FFT path (fft_path.cu) ----
// Vt[p1][p3][p2] = V(rev1[p1], rev2[p2], rev3[p3]) / N_r   (real type R)
qm_status launch_vt_prepare(qm_gspace g, const double* vloc, void* vt, bool fp32, cudaStream_t s);
// local + kinetic part for nb bands: out = kin*psi + (V psi)(G) (accumulate: out += ...);
// T = stick workspace; wait_k3 (may be NULL): event waited for before the first x-forward pass
qm_status launch_local_kinetic(qm_gspace g, int ik, int nb, const void* psi, int ld_psi,
                               const void* vt, void* out, int ld_out, void* tbuf,
                               size_t tbuf_bytes, bool fp32, cudaStream_t s,
                               cudaEvent_t wait_k3 = nullptr, bool accumulate = false, bool gamma = false);
size_t stick_buffer_bytes_per_band(qm_gspace g, int ik, bool fp32);

// The FFT path's tables of one k-point given by explicit device pointers (twiddles and kin
// in the precision of the call).
struct DevTables {
    int n[3];
    int ldx, ldy;
    AxisPlan plan[3];
    const void* tw[3];
    const int* rev[3];
    int nstick, nstick_pad, nrow;
    const int* stick_g0;
    const int* stick_plane;
    const int* rows;
    const int2* g_code;
    const void* kin;
};
qm_status launch_vt_prepare_tab(const DevTables& t, const double* vloc, void* vt, bool fp32, cudaStream_t s);
qm_status launch_local_kinetic_tab(const DevTables& t, int nb, const void* psi, int ld_psi, const void* vt,
                                   void* out, int ld_out, void* tbuf, size_t tbuf_bytes, bool fp32,
                                   cudaStream_t s);

// ---- complex GEMMs (zgemm.cu) ----
// C[m][n] = sum_k conj(A[m][k]) * B[n][k]   (A: M rows, B: N rows, k contiguous);
// split over K into `splits` partial sums reduced in a fixed order (deterministic).
qm_status zgemm_cn(int M, int N, int K, const double2* A, int lda, const double2* B, int ldb,
                   double2* C, int ldc, double2* partial, int splits, cudaStream_t s);
// C[m][n] (+)= alpha * sum_k A[k][m] * d[k] * B[k][n]   (d may be NULL -> 1)
qm_status zgemm_tn(int M, int N, int K, const double2* A, int lda, const double* d,
                   const double2* B, int ldb, double2* C, int ldc, bool accumulate,
                   cudaStream_t s, double alpha = 1.0);
int zgemm_cn_splits(int M, int N, int K);
// the same two products in double-FP32 arithmetic (FP64 in and out, products and sums on the
// FP32 pipe with error-free transformations, ~2^-46 relative accuracy): the precision form's
// FP64 phase
qm_status zgemm_cn_ds(int M, int N, int K, const double2* A, int lda, const double2* B, int ldb,
                      double2* C, int ldc, double2* partial, int splits, cudaStream_t s);
qm_status zgemm_tn_ds(int M, int N, int K, const double2* A, int lda, const double* d,
                      const double2* B, int ldb, double2* C, int ldc, bool accumulate,
                      cudaStream_t s, double alpha = 1.0);
// ---- tensor-core nonlocal step of the precision form (nonlocal_tc.cu) ----
constexpr int kMaxUmmaSplits = 64;
// out[b][g] (+)= sum_p beta[p][g] D_p <beta_p|psi_b> (FP32 complex in/out) as BF16x3 split
// tcgen05 products; err: device int set on a timed-out wait.
// The same product with operands pre-split into tile-blocked BF16 planes in global memory and
// streamed by bulk copies through a warp-specialised tcgen05 pipeline (nonlocal_tc.cu).
// beta_prepared: NULL (beta is split on every call, in `work`) or the output of
// nonlocal_tc_prepare (nonlocal_tc_beta_bytes bytes; depends on nproj and npw only).
// work: nonlocal_tc_bytes(nproj, nb, npw, beta_prepared == NULL) bytes.
qm_status nonlocal_tc(int nproj, int nb, int npw, const float2* beta, int ld_beta, const void* beta_prepared,
                      const float2* psi, int ld_psi, const double* D, float2* out, int ld_out, void* work, int* err,
                      cudaStream_t s, bool accumulate = false);
size_t nonlocal_tc_bytes(int nproj, int nb, int npw, bool with_beta);
size_t nonlocal_tc_beta_bytes(int nproj, int nb, int npw);
qm_status nonlocal_tc_prepare(int nproj, int nb, int npw, const float2* beta, int ld_beta, void* beta_work,
                              cudaStream_t s);
// qm_hpsi with the precision form's projectors optionally pre-split (beta_prepared, see
// nonlocal_tc); qm_hpsi itself passes NULL.  ds_nonlocal (QM_FP64 only): the nonlocal GEMMs in
// double-FP32 arithmetic (zgemm_cn_ds / zgemm_tn_ds), for the precision form's FP64 phase.
// gamma: the Gamma-point real-wavefunction FFT path (qm_hpsi_gamma; two bands per transform).
qm_status hpsi_run(qm_gspace g, int ik, int nb, const void* psi, int ld_psi, const double* vloc_r, int nproj,
                   const void* beta, int ld_beta, const void* beta_prepared, const double* D, void* out, int ld_out,
                   qm_precision prec, cudaStream_t s, bool ds_nonlocal = false, bool gamma = false);
// Subspace products of the Davidson FP32 phase on the tensor cores: FP64 storage rounded to
// FP32 on load, BF16x3 split products accumulated in FP32 per K split, splits summed in FP64.
//   cn: C[i][j] = sum_k conj(A[i][k]) B[j][k]                (as zgemm_cn)
//   tn: C[i][n] (+)= alpha sum_k A[k][i] B[k][n]             (as zgemm_tn with d = NULL)
// work: subspace_bf16x3_bytes(max M, max N) bytes; err: device int set on a timed-out wait
qm_status zgemm_cn_bf16x3(int M, int N, int K, const double2* A, int lda, const double2* B, int ldb,
                          double2* C, int ldc, void* work, size_t work_bytes, int* err, cudaStream_t s);
qm_status zgemm_tn_bf16x3(int M, int N, int K, const double2* A, int lda, const double2* B, int ldb,
                          double2* C, int ldc, bool accumulate, double alpha, void* work, size_t work_bytes,
                          int* err, cudaStream_t s);
size_t subspace_bf16x3_bytes(int max_m, int max_n);

// ---- learned preconditioner (mlp.cu) ----
// out_j(G) = K(f) R[sel[j]](G) for j < nu: the network's correction of the Davidson step;
// tk, eps: per band T_n and Ritz value; hdiag: the Hamiltonian's diagonal per plane wave (device);
// err: device int set on a timed-out wait
qm_status mlp_precond_apply(const float* theta, const double2* R, int ld, int npw, const int* sel, int nu,
                            const double* tk, const double* eps, const double* hdiag, const double* kin, double2* out,
                            int ldo, int* err, cudaStream_t s);
// hdiag[G] = T_G + mean(V) + sum_p D_p |beta_p(G)|^2 (FP64; work: kVmeanBlocks doubles)
constexpr int kVmeanBlocks = 256;
qm_status hamiltonian_diag(qm_gspace g, int ik, const double* vloc, int nproj, const double2* beta, int ld_beta,
                           const double* D, double* hdiag, double* work, cudaStream_t s);

// upper bound of the split-K partial buffer any gemm_cn call needs
size_t gemm_cn_partial_bytes(bool fp32);

// ---- dense FP64 subspace kernels (heev.cu, dense.cu) ----
// lowest nev eigenpairs of the Hermitian m x m matrix A (lda, destroyed): evals[nev] device,
// increasing; Y (m x nev, ld ldy) eigenvectors as columns; work heev_work_bytes(m, nev)
qm_status heev_lowest(double2* A, int lda, int m, int nev, double* evals, double2* Y, int ldy, void* work,
                      cudaStream_t s);
size_t heev_work_bytes(int m, int nev);
// Cholesky-with-dropping orthonormalisation: chol_transform factors S (nd x nd Gram matrix,
// destroyed) and counts the kept vectors into kept_dev; chol_transform_rows then writes the
// nd x kept transform W for gemm_tn.  keep, rank: nd ints; X: nd x nd scratch.
qm_status chol_transform(double2* S, int lds, int nd, double drop_rel, int* keep, int* rank, int* kept_dev,
                         double2* X, double2* W, int ldw_max, cudaStream_t s);
qm_status chol_transform_rows(const double2* L, int lds, int nd, const int* keep, const int* rank, int kept,
                              double2* X, double2* W, cudaStream_t s);

qm_status cgemm_cn(int M, int N, int K, const float2* A, int lda, const float2* B, int ldb,
                   float2* C, int ldc, float2* partial, int splits, cudaStream_t s);
qm_status cgemm_tn(int M, int N, int K, const float2* A, int lda, const double* d,
                   const float2* B, int ldb, float2* C, int ldc, bool accumulate,
                   cudaStream_t s, double alpha = 1.0);

}  // namespace qm
