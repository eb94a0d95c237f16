// Host-side engine: one context per structure, and a lockstep batch driver whose every
// kernel launch covers all structures still iterating.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/sgo.h"
#include "kernels.h"

namespace sgo {

struct Arena {
  char* base = nullptr;
  size_t used = 0, cap = 0;
  template <typename P>
  P* take(size_t count, size_t align = 256) {
    used = (used + align - 1) / align * align;
    P* p = reinterpret_cast<P*>(base + used);
    used += count * sizeof(P);
    return p;
  }
};

}  // namespace sgo

// One structure.  Owns all of its device memory.
struct sgo_ctx {
  // inputs
  double cell[9];
  std::vector<sgo_species> species;
  std::vector<int> spec;
  std::vector<double> pos;
  // projector list (host copy of the device arrays pj_*)
  std::vector<int> pj_atom, pj_kind, pj_first;
  std::vector<double> pj_d, pj_rp;
  double ecut = 0.0;
  int nb = 0;         // requested bands (occupied and reported)
  int nb_int = 0;     // bands the eigensolver carries: nb plus empty headroom (sgo_opts.extra_bands)
  sgo_opts opts;
  cudaStream_t stream = nullptr;
  int device = -1;    // the CUDA device current at sgo_create (owns every buffer)
  int precision = 0;  // 0 FP64, 1 mixed (FP32 wave data)
  // derived
  sgo::Prob d;        // descriptor (host copy, device pointers)
  int box_cols = 0;
  int ngbox_ew = 0;
  size_t tsize = 8;
  char* arena_setup = nullptr;
  char* arena_main = nullptr;
  bool warm = false;
  bool have_state = false;
  bool last_warm = false;   // the last evaluation started from the previous (or imported) state
  int last_iter = 0;
  double last_resid = 0.0;
  sgo_status last_status = SGO_OK;
  std::vector<double> h_scal, h_eps, h_occ, h_forces;
  int h_status[4] = {0, 0, 0, 0};
  // k-point mesh by zone folding (sgo_opts.kgrid): every field above describes the
  // kgrid[0] x kgrid[1] x kgrid[2] supercell; the caller's cell has nat_user atoms (the
  // supercell's first nat_user, translate t = 0) and lattice rows ucell
  int kgrid[3] = {1, 1, 1};
  int nk = 1;
  int nat_user = 0;
  double ucell[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  ~sgo_ctx();
};

namespace sgo {

// Lockstep driver over n contexts of the same precision.
class Engine {
 public:
  Engine(const std::vector<sgo_ctx*>& ctxs, cudaStream_t stream);
  ~Engine();
  bool ok() const { return ok_; }
  // Full evaluation: structure terms, SCF, optional forces.  per_item receives statuses.
  sgo_status run(bool want_forces, std::vector<sgo_status>* per_item);
  // Component calls on problem 0.
  sgo_status apply_h(const double* veff_c, int nvec, const double* psi, double* hpsi);
  sgo_status density(int nvec, const double* psi, const double* occ, double* rho);
  sgo_status export_density(double* rho);
  // warm-start state: rho_in(G) (complex, C order) and the packed wavefunctions
  sgo_status export_state(double* rho_g, double* psi);
  sgo_status import_state(const double* rho_g, const double* psi);
  sgo_status grid_transform(int sign, const double* in, double* out);
  sgo_status subspace(int nvec, const double* x, const double* y, double* c);
  sgo_status block_update(int nvec, const double* x, const double* m, double alpha, double beta, double* y);
  sgo_status structure_terms();
  // Live CUDA-event timing of one kernel class (see kTimerNames) over subsequent runs.
  bool timer_select(const char* name);
  void timer_read(double* ms, int* launches, double* bytes, double* flops);
  long long take_launches() {
    long long v = launches_;
    launches_ = 0;
    return v;
  }
  // Drive the SCF loop by captured CUDA graphs (batch engines); see build_graphs().
  void enable_graphs(bool on) { use_graph_ = on; }
  // Pick the GEMM tile knobs by timing candidates on this batch (see autotune()).
  void autotune();
  void tuning(int* out) const {
    out[0] = tc_kc_;
    out[1] = nn_tpc_;
    out[2] = tn_kc_;
  }
  // Batch evaluation with positions, energies, forces and statuses in device memory.
  sgo_status run_device(const double* pos, double* energies, double* forces, int* status);
  // Device-resident inputs and outputs of a batch evaluation, indexed by the member's
  // position in the whole batch (see set_slots).
  struct DeviceIO {
    const double* pos;
    double* energies;
    double* forces;
    int* status;
  };
  // Position of each member of this engine in the whole batch and the offset (doubles) of
  // its 3 natom coordinates in the batch's packed position and force arrays.
  bool set_slots(const std::vector<int>& slot, const std::vector<int>& foff);
  // run() in four steps, so that the engines of several sub-batches overlap on the GPU:
  // enter() orders the engine's private stream after the caller's, launch() enqueues the
  // whole evaluation (in graph mode without any host wait), leave() orders the caller's
  // stream after it, finish() waits for it and reads the results back.  Without graphs
  // (or with the live timer) the work runs on the caller's stream and launch() waits on
  // the host once per SCF iteration.
  sgo_status enter();
  sgo_status launch(bool want_forces, const DeviceIO* io);
  void leave();
  sgo_status finish(std::vector<sgo_status>* per_item);
  int size() const { return n_; }

 private:
  template <typename T> sgo_status launch_t(bool want_forces);
  template <typename T> void scf_iteration(int ncg, bool count_iter);
  template <typename T> void density_energy(int mode);
  template <typename T> void polish();
  template <typename T> bool build_polish_graphs();
  bool read_active();
  void pulay_step();
  template <typename T> bool build_graphs();
  template <typename T> void hpsi(int src, int dst);
  template <typename T> void rayleigh_ritz(bool rotate_history);
  template <typename T> void cg_step();
  template <typename T> void davidson_step();
  template <typename T> void eig_step() { davidson_ ? davidson_step<T>() : cg_step<T>(); }
  void rr_solve(int blk);
  template <typename T> void tn(int akind, int arole, int bkind, int brole, int dst, bool allow_tc = true);
  template <typename T>
  void nn(int akind, int arole, int msel, int yrole, double alpha, double beta, bool image_ready = false);
  template <typename T>
  void nn_pairs(int akind, const RolePairs& rp, int msel, double alpha, double beta, bool image_ready);
  template <typename T> void rotate_pairs(const RolePairs& rp, const RolePairs& swap);
  int work_mult_ = 1;  // operand pairs of the NN launch being timed
  void grid_fft(int which, int sign, bool fp32 = false);
  template <typename T> void grid_fft_raw(int which, int sign);
  void potential();
  void energies_at_rho_out(bool count_iter);
  void pulay();
  void sync_active();
  void set_scal(int idx, double v, bool only_active);
  void tbeg(int kind);
  void tend(int kind);
  void work_of(int kind, double* bytes, double* flops) const;
  int timer_kind_ = -1;
  mutable long long launches_ = 0;  // kernel launches issued (one per Launch built)
  std::vector<cudaEvent_t> ev_;
  std::vector<double> ev_bytes_, ev_flops_;
  int ev_used_ = 0;
  double t_ms_ = 0.0, t_bytes_ = 0.0, t_flops_ = 0.0;
  int t_launches_ = 0;
  void swap_roles(int a, int b);
  Launch L(const WorkMap& m) const;
  WorkMap make_map(const std::vector<int>& counts);

  std::vector<sgo_ctx*> ctx_;
  int n_ = 0;
  cudaStream_t stream_;
  int precision_ = 0;
  bool ok_ = false;
  Prob* d_probs_ = nullptr;
  int* d_active_ = nullptr;
  std::vector<int> h_active_;
  std::vector<void*> allocs_;
  int max_n1_ = 0, max_n2_ = 0, max_n3_ = 0, max_n12_ = 0, max_nb_ = 0, plane_threads_ = 128;
  WorkMap m_zcol_, m_plane_, m_dens_, m_gz_, m_gp_, m_gew_, m_gch_, m_bands_, m_tn_ww_, m_tn_bw_, m_tn_dw_,
      m_red_ww_, m_red_bw_, m_red_dw_, m_nn_, m_atoms_, m_projs_, m_atomch_, m_ewsg_, m_prob_, m_tc_, m_nntc_;
  WorkMap m_preg_[2], m_dreg_[2], m_zreg_[2];  // register-FFT plane / column kernels, per size class
  size_t preg_smem_[2] = {0, 0}, dreg_smem_[2] = {0, 0}, zreg_smem_[2] = {0, 0};
  WorkMap m_ppair_, m_dpair_, m_zpair_;         // lane-pair register FFT kernels (lengths 96-128)
  size_t ppair_smem_ = 0, dpair_smem_ = 0, zpair_smem_ = 0;
  WorkMap m_gx_, m_gy_;                         // FP64 grid transforms of planes too large for one CTA
  WorkMap m_bigy_, m_bigx_, m_bigdy_, m_bigd_;  // plane passes by line blocks (big planes)
  template <typename T> void wave_to_cols(int src);
  template <typename T> void cols_to_wave(int src, int dst);
  bool tc_ok_[3] = {false, false, false};      // TN on tcgen05, per A-operand kind
  bool nn_tc_ok_[3] = {false, false, false};   // NN on tcgen05, per X-operand kind
  void* d_tmaps_ = nullptr;                    // [n][TC_NSLOT][TC_NMAPKIND] tensor maps
  float* d_nnimg_ = nullptr;                   // [n][nnimg_stride_] NN B-operand images
  size_t nnimg_stride_ = 0;
  int nnimg_max_[3] = {0, 0, 0};
  double* d_part_ = nullptr;
  size_t part_stride_ = 0;
  double* d_gpart_ = nullptr;
  int maxchunk_ = 1;
  bool rr_smem_ = true;
  bool rr_f32_ = false;
  bool rr_cluster_ = false;          // subspace too large for one CTA: cluster eigensolve
  bool davidson_ = false;            // block Davidson steps (2 n_b Rayleigh-Ritz) instead of CG
  bool gga_ = false;                 // PBE exchange-correlation
  double cg_adapt_ = 0.0;            // density residual above which the last CG step is left out
  int* d_saved_ = nullptr;           // active mask kept across that step
  int rr_n_ = 0;                     // largest subspace of one Rayleigh-Ritz call
  unsigned char* d_rrc_ = nullptr;   // its per-member global scratch
  size_t rrc_stride_ = 0;
  unsigned char* d_rr1_ = nullptr;   // one-CTA eigensolve beyond shared memory: global scratch
  size_t rr1_stride_ = 0;            // bytes per member
  size_t rr_smem_bytes_ = 0;
  double* d_flags_ = nullptr;   // [n][4] gathered per iteration
  // pinned read-back area (device-to-host copies into it do not block the host):
  // hp_ = flags [n][4], then per member scal, eps, occ, forces at hp_off_[p];
  // hpi_ = iteration count, then per member status[4]
  double* hp_ = nullptr;
  int* hpi_ = nullptr;
  std::vector<size_t> hp_off_;
  int* d_slot_ = nullptr;       // [n] member's position in the whole batch
  int* d_foff_ = nullptr;       // [n] offset of its coordinates in the batch's arrays
  // state of the evaluation between launch() and finish()
  cudaStream_t user_stream_ = nullptr, run_stream_ = nullptr;
  bool run_graph_ = false, run_forces_ = false;
  int run_nonsc_ = 0, run_it_ = 0, run_na_ = 0;
  sgo_status run_status_ = SGO_OK;
  // graph mode: captured iterations, the device iteration counter, a private stream (the
  // caller's may be the legacy default stream, which cannot be captured)
  bool use_graph_ = false;
  // GEMM tile knobs: K chunk of the tensor-core TN, 128-wave tiles per NN CTA, K chunk of
  // the CUDA-core TN; the maps that depend on them
  int tc_kc_ = TC_KC, nn_tpc_ = NN_TPC, tn_kc_ = TN_KC;
  void build_gemm_maps();
  cudaGraphExec_t g_nonscf_ = nullptr, g_scf_ = nullptr;
  // the residual-controlled CG steps after the SCF stopping rule (a WHILE node whose body
  // is one step) and the density and energy of the refined bands
  cudaGraphExec_t g_polish_ = nullptr, g_tail_ = nullptr;
  long long graph_launches_[4] = {0, 0, 0, 0};
  int* d_iter_ = nullptr;       // [2]: SCF iterations, residual-controlled loop passes
  long long wait_ns_ = 2000000000LL;  // watchdog of the tensor-core kernels' waits
  int rr_cap_ = 10;             // Jacobi sweep cap of the FP32 subspace eigensolve
  cudaStream_t own_stream_ = nullptr;
  cudaEvent_t ev_in_ = nullptr, ev_out_ = nullptr;
};

// Kernel classes the engine can time live (CUDA events on its stream).
enum {
  TK_PLANE_VPSI = 0, TK_WAVE_TO_COLS, TK_COLS_TO_WAVE, TK_PLANE_DENSITY, TK_GEMM_TN, TK_GEMM_NN, TK_RR,
  TK_GRID_FFT, TK_CG_BAND, TK_GRID_OTHER, TK_GEMM_SMALL, TK_COUNT
};
extern const char* const kTimerNames[TK_COUNT];

// Kernel choice of the plane passes of one structure (see plane_paths in engine.cu).
struct PlanePaths {
  bool preg = false, dreg = false, ppair = false, dpair = false, psmem = false, pbig = false, dbig = false;
};
PlanePaths plane_paths(const Prob& d, int precision);

// Device memory of the library: cudaMalloc, or the caller's allocator when one is installed
// (sgo_set_allocator); dev_free returns a block to whichever allocator gave it.
void set_allocator(sgo_alloc_fn a, sgo_free_fn f, void* user);
cudaError_t dev_malloc_bytes(void** p, size_t bytes, cudaStream_t s = nullptr);
template <typename P>
cudaError_t dev_malloc(P** p, size_t bytes, cudaStream_t s = nullptr) {
  void* v = nullptr;
  const cudaError_t e = dev_malloc_bytes(&v, bytes, s);
  *p = static_cast<P*>(v);
  return e;
}
void dev_free(void* p, bool synced = false);  // synced: the device was synchronised already

// Context set-up (basis on the device, allocation, tables).  Returns status.
sgo_status ctx_setup(sgo_ctx* c);
sgo_status set_positions(sgo_ctx* c, const double* pos);

}  // namespace sgo
