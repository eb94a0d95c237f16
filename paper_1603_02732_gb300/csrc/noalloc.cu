// H.psi without any device allocation in the call (sgo_apply_hamiltonian_noalloc).
//
// Some applications cannot let a library allocate device memory while they run: a host
// process that has handed all device memory to its own pool allocator, one that works
// under a fixed memory budget, or a latency-critical loop that cannot afford the implicit
// synchronisation and unpredictable latency of cudaMalloc/cudaFree.  For them this
// entry point computes the same H.psi as sgo_apply_hamiltonian using only memory that
// already exists: the context's buffers (allocated once by sgo_create) and one
// file-scope device array, g_noalloc_scratch, which holds the launch descriptors, the
// split-K partial sums of the projector overlaps and the staged inputs and outputs.
//
// The array lives on every GPU that loads the library until the process exits.  In host
// code its name is only a host-side stand-in, so its device address is looked up with
// cudaGetSymbolAddress, once per device, with that device current, on the first call made
// on that device; that first call should come before any stream capture.  The device
// current at a call must be the context's (the one current at sgo_create).  Every call
// shares the array and leaves its contents behind; each call writes every byte it later
// reads, so nothing has to be cleared.  Calls that overlap on the GPU (different streams
// or threads) race on the array.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "engine.h"

namespace sgo {
const char* last_error();
}

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB per GPU
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
void* g_addr[kMaxDevices] = {nullptr};

int div_up(long a, long b) { return (int)((a + b - 1) / b); }

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// The array's address on the context's device.  The address is looked up with the
// current device, so that device must be the one whose memory holds the context (and on
// which its stream runs): a context used with another device current is refused.
sgo_status scratch_address(const sgo_ctx* c, void** out) {
  int dev = 0;
  if (!sgo::cuda_ok(cudaGetDevice(&dev), "cudaGetDevice")) return SGO_ERR_CUDA;
  if (dev != c->device) {
    sgo::set_error("no-alloc call with device " + std::to_string(dev) + " current, but the context lives on device " +
                   std::to_string(c->device));
    return SGO_ERR_ARG;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    sgo::set_error("device ordinal beyond the no-alloc address cache");
    return SGO_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (!sgo::cuda_ok(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress(g_noalloc_scratch)"))
      return SGO_ERR_CUDA;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return SGO_OK;
}

template <typename T>
sgo_status run(sgo_ctx* c, const double* veff, int nvec, const double* psi, double* hpsi, char* base) {
  using namespace sgo;
  const Prob& d = c->d;
  cudaStream_t st = c->stream;
  const int nsplit = div_up(d.npw, TN_KC);
  const size_t part_stride = (size_t)nsplit * d.nproj * d.nb;
  // layout of the scratch array
  size_t off = 0;
  const size_t o_prob = off;
  off = align256(off + sizeof(Prob));
  const size_t o_act = off;
  off = align256(off + sizeof(int));
  enum { M_ZCOL = 0, M_PLANE, M_BANDS, M_ATOMS, M_TN, M_RED, M_NN, M_GEW, M_PROJ, NMAP };
  const size_t o_maps = off;
  off = align256(off + sizeof(int) * 2 * NMAP);
  const size_t o_part = off;
  off = align256(off + sizeof(double) * part_stride);
  const size_t o_veff = off;
  off = align256(off + sizeof(double) * d.ngrid);
  const size_t o_psi = off;
  off = align256(off + sizeof(double) * (size_t)nvec * d.npw);
  const size_t o_out = off;
  off = align256(off + sizeof(double) * (size_t)nvec * d.npw);
  // this path runs the shared-memory plane engine only (two whole planes per CTA)
  if ((size_t)(2 * d.n1 * d.n2 + d.n1 + d.n2) * sizeof(cplx<T>) > 220 * 1024) {
    set_error("FFT planes too large for the no-alloc path (two whole planes per CTA in shared memory)");
    return SGO_ERR_ARG;
  }
  if (off > kNoAllocScratchBytes) {
    set_error("problem too large for the no-alloc scratch: needs " + std::to_string(off) + " bytes, limit " +
              std::to_string(kNoAllocScratchBytes));
    return SGO_ERR_ARG;
  }
  const int counts[NMAP] = {d.npair * div_up(d.ncp, QCP), d.npair * d.n3, d.nb, d.natom,
                            div_up(d.nproj, TN_TILE) * div_up(d.nb, TN_TILE) * nsplit, div_up(d.nproj * d.nb, 256),
                            div_up(d.npw, 64 * NN_RT) * div_up(d.nb, 64), div_up(d.ngrid, GRID_EW_POINTS), d.nproj};
  int maps[2 * NMAP];
  for (int i = 0; i < NMAP; ++i) {
    maps[2 * i] = 0;
    maps[2 * i + 1] = counts[i];
  }
  Prob h = d;
  for (int i = 0; i < NWB; ++i) h.role[i] = i;
  const int one = 1;
  if (!cuda_ok(cudaMemcpyAsync(base + o_prob, &h, sizeof(Prob), cudaMemcpyHostToDevice, st), "stage descriptor") ||
      !cuda_ok(cudaMemcpyAsync(base + o_act, &one, sizeof(int), cudaMemcpyHostToDevice, st), "stage mask") ||
      !cuda_ok(cudaMemcpyAsync(base + o_maps, maps, sizeof(maps), cudaMemcpyHostToDevice, st), "stage maps") ||
      !cuda_ok(cudaMemcpyAsync(base + o_veff, veff, sizeof(double) * d.ngrid, cudaMemcpyHostToDevice, st),
               "stage veff") ||
      !cuda_ok(cudaMemcpyAsync(base + o_psi, psi, sizeof(double) * (size_t)nvec * d.npw, cudaMemcpyHostToDevice, st),
               "stage psi"))
    return SGO_ERR_CUDA;
  const Prob* dprob = reinterpret_cast<const Prob*>(base + o_prob);
  const int* dact = reinterpret_cast<const int*>(base + o_act);
  const int* dmaps = reinterpret_cast<const int*>(base + o_maps);
  auto launch = [&](int m) {
    Launch l;
    l.ka = KArgs{dprob, dmaps + 2 * m, 1, dact};
    l.map.start = const_cast<int*>(dmaps + 2 * m);
    l.map.total = counts[m];
    l.map.maxper = counts[m];
    l.stream = st;
    l.max_n1 = d.n1;
    l.max_n2 = d.n2;
    l.max_n3 = d.n3;
    l.max_n12 = d.n1 * d.n2;
    l.max_nb = d.nb;
    l.plane_threads = PLANE_THREADS;
    return l;
  };
  fft_set_smem_limits(220 * 1024);
  linalg_set_smem_limits(220 * 1024);
  double* part = reinterpret_cast<double*>(base + o_part);
  double* dpsi = reinterpret_cast<double*>(base + o_psi);
  double* dout = reinterpret_cast<double*>(base + o_out);
  launch_phases(launch(M_ATOMS));
  launch_build_projectors<T>(launch(M_PROJ), 0);
  launch_veff<T>(launch(M_GEW), reinterpret_cast<const double*>(base + o_veff));
  launch_copy_in<T>(launch(M_BANDS), WB_W, dpsi, nvec);
  launch_wave_to_cols<T>(launch(M_ZCOL), WB_W);
  launch_plane_vpsi<T>(launch(M_PLANE));
  launch_cols_to_wave<T>(launch(M_ZCOL), WB_W, WB_W2);
  launch_gemm_tn<T>(launch(M_TN), OPK_B, 0, OPK_WB, WB_W, part, part_stride);
  launch_gemm_tn_reduce(launch(M_RED), OPK_B, OPK_WB, DD_PROJ, part, part_stride);
  launch_gemm_nn<T>(launch(M_NN), OPK_B, role_pair(0, WB_W2), DD_PROJ_D, 1.0, 1.0);
  launch_copy_out<T>(launch(M_BANDS), WB_W2, dout, nvec);
  if (!cuda_ok(cudaGetLastError(), "no-alloc H.psi launch") ||
      !cuda_ok(cudaMemcpyAsync(hpsi, dout, sizeof(double) * (size_t)nvec * d.npw, cudaMemcpyDeviceToHost, st),
               "read hpsi") ||
      !cuda_ok(cudaStreamSynchronize(st), "no-alloc H.psi"))
    return SGO_ERR_CUDA;
  return SGO_OK;
}

}  // namespace

extern "C" SGO_API sgo_status sgo_apply_hamiltonian_noalloc(sgo_ctx* c, const double* veff, int nvec,
                                                            const double* psi, double* hpsi) {
  if (!c || !veff || !psi || !hpsi || nvec < 1 || nvec > c->nb) return SGO_ERR_ARG;
  void* base = nullptr;
  sgo_status s = scratch_address(c, &base);
  if (s != SGO_OK) return s;
  return c->precision ? run<float>(c, veff, nvec, psi, hpsi, static_cast<char*>(base))
                      : run<double>(c, veff, nvec, psi, hpsi, static_cast<char*>(base));
}
