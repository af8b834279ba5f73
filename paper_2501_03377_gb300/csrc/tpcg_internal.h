// Internal declarations of libtpcg (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <map>
#include <vector>

#include "../../include/tpcg.h"

namespace tpcg {

constexpr int kBcP = 0, kBcD = 1, kBcN = 2, kBcDN = 3, kBcND = 4;

// FP64 eigenpairs of one axis (Algorithm 5).  lam is divided by h^2.
struct AxisBasis {
  int len = 1;
  int bc = 0;
  double h = 1.0;
  std::vector<double> lam;  // len
  std::vector<double> V;    // len*len row-major, column k = eigenvector k
  double orth_err = 0.0, recon_err = 0.0;
};

std::vector<double> lap1d_dense(int n, int bc);
void closed_form_eigenpairs(int n, int bc, std::vector<double>& lam, std::vector<double>& V);
void eigen_check(int n, int bc, const std::vector<double>& lam, const std::vector<double>& V, double* orth_err,
                 double* recon_err);
int build_axis(int len, int bc, double h, AxisBasis& ax);

// One mode-product pass of Algorithm 7: for every row r = a*B + b of the
// input (an A x B x C array with C contiguous, rows in_pitch elements apart)
//     out[a*oa + b*ob + c'*oc] = sum_c X[r][c] * Wm[c][c']   (W = V or V^T),
// optionally multiplied by the Hadamard pseudoinverse G (Algorithm 7).  The output
// strides place the next contraction index contiguously, so every pass
// contracts a contiguous index.
struct StageParams {
  int A, B, C, Cout;
  int in_pitch;
  long long oa, ob, oc;
  int axis;        // 0 x, 1 y, 2 z
  int dir;         // 0 forward (W = V), 1 backward (W = V^T)
  int scale;       // apply G
  int lamA, lamB, lamC;  // axis whose eigenvalue index is a / b / c'
  int final_stage;
  int out_pitch_elems;   // row pitch of the output viewed as the next stage's input
  int out_rows;          // rows of the output viewed as the next stage's input
  int out_C;             // contiguous extent of that view
};

struct SolveState;  // device-side scalars (tpcg_dev.cuh)

// Kernel kinds for the launch counter and the optional event profiler.
// Persistent fixed-point sweeps (grid size per kernel, from its occupancy).
enum FxKernel { kFxDir = 0, kFxUpd, kFxTrue, kFxInit, kFxCount };

enum KernelKind {
  kKEtaSum = 0, kKInit, kKDirection, kKUpdate, kKTrueRes, kKCenter, kKApply, kKModeF64, kKModeTC, kKConvert, kKFormU,
  kKindCount
};
const char* kernel_kind_name(int kind);

// Optional per-launch CUDA-event timing (tpcg_profile_begin / _end).
struct Profiler {
  bool on = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> recs;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  unsigned long long launches[kKindCount] = {};
  double ms[kKindCount] = {};
  unsigned long long timed[kKindCount] = {};
};

// One PCG solve driven as a resumable job: job_start() enqueues the set-up
// (Algorithm 1 set-up) and the first chunk of iterations; whenever the
// plan's state event has completed, job_step() inspects the device state and
// enqueues the next chunk or the exit work.  Many jobs on different plans (and
// streams) can be driven by one host thread.
struct SolveJob {
  tpcg_plan* p = nullptr;
  const double* eta = nullptr;
  double* ups = nullptr;
  double tol = 1e-10;
  int maxit = 100;
  unsigned flags = 0;
  int issued = 0, chunk = 0;
  int phase = 0;  // 0 not started, 1 iterating, 2 finishing, 3 finished
  int done_host = 0, status_host = 0;
  int status = 0;
  tpcg_info info{};
};
// A launch sequence of a solve captured as a CUDA graph: the set-up (what = 0) or a chunk of `count`
// iterations starting at iteration k0 (what = 1); flags: zero initial guess and the 16-byte alignment of
// the caller's arrays (they choose kernel variants); gen: the plan's option generation.
struct GraphKey {
  int what, k0, count;
  unsigned flags, gen;
  bool operator<(const GraphKey& o) const {
    if (what != o.what) return what < o.what;
    if (k0 != o.k0) return k0 < o.k0;
    if (count != o.count) return count < o.count;
    if (flags != o.flags) return flags < o.flags;
    return gen < o.gen;
  }
};
struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  unsigned long long kernels = 0;  // kernel launches the sequence holds (the plan's launch count)
  unsigned long long used = 0;     // last use (eviction order)
};

int job_start(SolveJob& j);
bool job_ready(const SolveJob& j);
int job_step(SolveJob& j);
void graph_reset(tpcg_plan* p);

}  // namespace tpcg

struct tpcg_plan {
  int nx = 0, ny = 0, nz = 0;
  int bc[3] = {0, 0, 0};
  double h[3] = {1, 1, 1};
  int prec = TPCG_FP64;
  cudaStream_t stream = nullptr;
  bool singular = false;
  bool is2d = false;
  long long N = 0;
  int device = 0;
  int num_sms = 0;
  tpcg::AxisBasis ax[3];

  // device: eigenbases
  double* d_W64[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};  // [axis][dir] FP64 W = V or V^T
  double* d_lam64[3] = {nullptr, nullptr, nullptr};
  float* d_lam32[3] = {nullptr, nullptr, nullptr};
  void* d_Wt16[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};   // [axis][dir] BF16 W^T (K-major)
  int pitch16[3] = {0, 0, 0};   // row pitch (elements) of BF16 arrays whose contiguous extent is axis l

  // device: PCG workspaces
  double* d_R = nullptr;
  void* d_P[8] = {};  // directions: FP64 ping-pong [0..1], or the mixed forms' ring of int32 fixed point
                     // (one allocation, d_P[0] its base; p_slots slots)
  int p_slots = 2;   // mixed forms: 2 (in-place update), kPRing once TPCG_OPT_DEFER_U has been set
  double* d_W = nullptr;               // W = L P (FP64 form only)
  void* d_Z = nullptr;       // FP64 (FP64 form) or FP32 (mixed forms)
  void* d_Rlp = nullptr;     // tensor-core copy of R (mixed forms), row pitch pitch16[0]
  int lp_kind = 0;           // 0 none (FP64 form), 1 BF16, 2 FP16 scaled by 2^lp_shift, 3 TF32 (FP32
                             // containers), 4 BF16 hi/lo pair (two planes of 16-bit words)
  size_t lp_plane = 0;       // kind 4: 16-bit words from the hi plane of d_Rlp to its lo plane
  void* d_T[2] = {nullptr, nullptr};  // mode-product intermediates
  size_t t_elems = 0;
  size_t t_plane = 0;        // kind 4: 16-bit words from the hi plane of a d_T buffer to its lo plane
  double* d_eta_h = nullptr;  // device copies for tpcg_solve_host
  double* d_ups_h = nullptr;
  // tpcg_solve_host_stream: the second slot of its two-slot pipeline (the first is d_eta_h / d_ups_h),
  // its copy streams and its per-slot events (all created on first use)
  double* d_eta_h2 = nullptr;
  double* d_ups_h2 = nullptr;
  cudaStream_t s_in = nullptr, s_out = nullptr;
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_solved[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
  tpcg::SolveState* d_state = nullptr;
  tpcg::SolveState* h_state = nullptr;  // pinned
  cudaEvent_t ev_state = nullptr;        // recorded after each read-back of the device state
  double* d_partials = nullptr;
  size_t partial_slots = 0;
  int* d_err = nullptr;   // device error word of bounded waits

  std::vector<tpcg::StageParams> stages;
  void* tc_state = nullptr;   // tensor-core pass descriptors (tensor maps, launch shapes)
  void* slab_state = nullptr; // frontal-slice launch descriptors (3D grids where they apply)
  mutable unsigned long long launch_count = 0;   // kernels launched by this plan
  mutable tpcg::Profiler prof;
  size_t device_bytes = 0;

  // launch configuration (fixed per plan so that reductions are reproducible)
  dim3 st_grid, st_block;   // stencil kernels
  int st_zchunk = 1;
  int sweep_grain = 4;  // TPCG_OPT_SWEEP_GRAIN: least (tile, plane) pairs (x 256 points) per sweep block
  int fx_blocks[tpcg::kFxCount] = {1, 1, 1, 1};  // FxKernel -> blocks of the persistent fixed-point sweeps
  // comparator preconditioner of the FP64 form (TPCG_PRECOND_*), Jacobi(p, omega) and its table of
  // 1 / (omega d) indexed by the boundary class (start, interior, end) of x + 3 y + 9 z
  int pc_kind = 0;
  int jac_p = 3;
  double jac_omega = 1.3;
  double jac_invd[27] = {};
  int stream_blocks = 0;    // streaming kernels
  int defer_u = 0;          // mixed forms: TPCG_OPT_DEFER_U (U += alpha P recorded, applied by k_form_u)
  int tc_fuse = 1;          // mixed forms: TPCG_OPT_FUSE_G (the two passes around G in one launch)
  int tc_slab = 1;          // mixed forms: TPCG_OPT_SLICES (frontal-slice launches where they apply)
  int last_iters = 0;      // iterations of the plan's previous converged solve (first chunk of the next)
  // TPCG_OPT_GRAPHS: the solve's launch sequences captured as CUDA graphs on first use and replayed
  int use_graphs = 0;
  unsigned graph_gen = 0;               // bumped whenever an option or buffer the sequences hold changes
  unsigned long long graph_clock = 0;
  std::map<tpcg::GraphKey, tpcg::GraphEntry> graphs;
};
