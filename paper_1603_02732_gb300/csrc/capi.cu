// extern "C" boundary of the engine (declarations and contracts in include/sgo.h).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <thread>
#include <cstring>
#include <memory>
#include <new>

#include "engine.h"

namespace sgo {
const char* last_error();
}
// relax.cpp (library-internal)
extern "C" int sgo_relax_natoms(const sgo_relax* r);

struct sgo_batch {
  std::vector<sgo_ctx*> ctxs;
  // one engine per sub-batch; members[e] = positions in ctxs of engine e's members
  std::vector<std::unique_ptr<sgo::Engine>> engs;
  std::vector<std::vector<int>> members;
};

namespace {

sgo::Engine* solo_engine(sgo_ctx* c) {
  // A context's own engine (batch of one); rebuilt on every call (cheap: a few small maps).
  return new sgo::Engine(std::vector<sgo_ctx*>{c}, c->stream);
}

// Number of sub-batches: the caller's choice, else (graph mode) three from 24 members on and
// two from 16, so that the latency-bound kernels of one sub-batch (the subspace eigensolve,
// the small GEMMs, the per-band vector kernels) overlap the others' large ones.  On the
// 64-member population, measured: 1, 2, 3, 4 sub-batches give 190, 203, 213, 211 evals/s.
int sub_batch_count(int n, const sgo_opts& o) {
  int k = o.sub_batches;
  if (k <= 0) k = n >= 24 ? 3 : n >= 16 ? 2 : 1;
  if (!o.graph) k = 1;
  return std::max(1, std::min(k, n));
}

// Split the members into k sub-batches of about equal work (longest job first onto the
// least loaded sub-batch); the work of a member is taken as n_b (N_grid log N_grid + n_b N_pw),
// its FFT and subspace GEMM terms.  Members keep their batch order inside a sub-batch.
std::vector<std::vector<int>> split_members(const std::vector<sgo_ctx*>& ctxs, int k) {
  const int n = (int)ctxs.size();
  std::vector<double> cost(n);
  for (int i = 0; i < n; ++i) {
    const double ng = (double)ctxs[i]->d.ngrid, nb = ctxs[i]->d.nb;
    cost[i] = nb * (ng * std::log2(std::max(2.0, ng)) + nb * (double)ctxs[i]->d.npw);
  }
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<double> load(k, 0.0);
  std::vector<std::vector<int>> out(k);
  for (int i : order) {
    const int e = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[e] += cost[i];
    out[e].push_back(i);
  }
  for (auto& v : out) std::sort(v.begin(), v.end());
  return out;
}

// Run every sub-batch: all enter first (so that none is ordered after another's end), then
// all launch, all leave, all finish.
sgo_status run_batch(sgo_batch* b, const sgo::Engine::DeviceIO* io, std::vector<sgo_status>* per_item) {
  sgo_status err = SGO_OK;
  for (auto& e : b->engs)
    if (e->enter() == SGO_ERR_CUDA) err = SGO_ERR_CUDA;
  for (auto& e : b->engs)
    if (e->launch(true, io) == SGO_ERR_CUDA) err = SGO_ERR_CUDA;
  for (auto& e : b->engs) e->leave();
  for (size_t k = 0; k < b->engs.size(); ++k) {
    std::vector<sgo_status> st(b->engs[k]->size(), SGO_OK);
    if (b->engs[k]->finish(&st) == SGO_ERR_CUDA) err = SGO_ERR_CUDA;
    if (per_item)
      for (size_t j = 0; j < st.size(); ++j) (*per_item)[b->members[k][j]] = st[j];
  }
  return err;
}

// Zone folding (sgo_opts.kgrid): the supercell's atoms are the caller's, translated by
// t . A for every t = (t1, t2, t3), t_i < kgrid[i], t-major (t = 0 first).
void expand_positions(const int kgrid[3], const double* ucell, int nat, const double* pos, double* out) {
  int t = 0;
  for (int t1 = 0; t1 < kgrid[0]; ++t1)
    for (int t2 = 0; t2 < kgrid[1]; ++t2)
      for (int t3 = 0; t3 < kgrid[2]; ++t3, ++t)
        for (int a = 0; a < nat; ++a)
          for (int x = 0; x < 3; ++x)
            out[(size_t)(t * nat + a) * 3 + x] =
                pos[3 * a + x] + t1 * ucell[x] + t2 * ucell[3 + x] + t3 * ucell[6 + x];
}

// The caller's positions into the context (expanded over the translates of a k-point
// context).
sgo_status set_user_positions(sgo_ctx* c, const double* pos) {
  if (c->nk == 1) return sgo::set_positions(c, pos);
  std::vector<double> big((size_t)3 * c->nat_user * c->nk);
  expand_positions(c->kgrid, c->ucell, c->nat_user, pos, big.data());
  return sgo::set_positions(c, big.data());
}

// The free energy per cell of the caller and the forces on its atoms: the supercell's
// divided by the number of translates, resp. averaged over the translates of each atom
// (equal up to rounding: the supercell is periodic in the caller's cell).
double user_energy(const sgo_ctx* c) { return c->h_scal[sgo::SC_FREE] / c->nk; }
void user_forces(const sgo_ctx* c, double* out) {
  const size_t n = (size_t)3 * c->nat_user;
  if (c->nk == 1) {
    std::memcpy(out, c->h_forces.data(), sizeof(double) * n);
    return;
  }
  for (size_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int t = 0; t < c->nk; ++t) s += c->h_forces[t * n + i];
    out[i] = s / c->nk;
  }
}

}  // namespace

extern "C" {

sgo_status sgo_set_allocator(sgo_alloc_fn alloc, sgo_free_fn release, void* user) {
  if ((alloc == nullptr) != (release == nullptr)) {
    sgo::set_error("sgo_set_allocator needs both functions or neither");
    return SGO_ERR_ARG;
  }
  sgo::set_allocator(alloc, release, user);
  return SGO_OK;
}

void sgo_opts_default(sgo_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = 0;
  o->kT = 0.0;
  o->scf_tol_e = 1e-8;
  o->scf_tol_rho = 1e-7;
  o->max_scf = 100;
  o->pulay_hist = 8;
  o->mix_alpha = 0.5;
  o->kerker_q0 = 0.8;
  o->ncg = 2;
  o->ncg_first = 6;
  o->n_nonscf = 0;
  o->seed = 12345ull;
  o->gemm_tc = 1;
  o->graph = 1;
  o->autotune = 1;
  o->eig_tol = 1e-4;
  o->max_polish = 40;
  o->rr_fp64 = 0;
  o->watchdog_ms = 0.0;
  o->extra_bands = -1;
  o->rr_cluster = -1;
  o->eigensolver = 0;
  o->xc = 0;
  o->cg_adapt = 0.0;
  o->kgrid[0] = o->kgrid[1] = o->kgrid[2] = 1;
}

sgo_status sgo_create(const double cell[9], int nspecies, const sgo_species* sp, int natoms, const int* species_of_atom,
                      const double* pos, double ecut, int nbands, const sgo_opts* o, void* cuda_stream,
                      sgo_ctx** out) {
  if (!out) return SGO_ERR_ARG;
  *out = nullptr;
  if (!cell || !sp || !species_of_atom || !pos || nspecies < 1 || nspecies > sgo::MAX_SPECIES || natoms < 1 ||
      !(ecut > 0.0) || nbands < 1) {
    sgo::set_error("invalid argument");
    return SGO_ERR_ARG;
  }
  sgo_ctx* c = new (std::nothrow) sgo_ctx();
  if (!c) return SGO_ERR_OOM;
  if (o) c->opts = *o;
  else sgo_opts_default(&c->opts);
  // a k mesh: the context becomes the kgrid supercell (rows kgrid[i] a_i, the atoms of every
  // translate, kgrid[0] kgrid[1] kgrid[2] times the bands, a given FFT grid scaled per axis)
  long long nk = 1;
  for (int i = 0; i < 3; ++i) {
    c->kgrid[i] = std::max(1, c->opts.kgrid[i]);
    c->opts.kgrid[i] = c->kgrid[i];
    nk *= c->kgrid[i];
  }
  if (nk > 4096 || (long long)natoms * nk > 100000 || (long long)nbands * nk > 100000) {
    delete c;
    sgo::set_error("k mesh too large for zone folding");
    return SGO_ERR_ARG;
  }
  c->nk = (int)nk;
  c->nat_user = natoms;
  std::memcpy(c->ucell, cell, sizeof(double) * 9);
  for (int i = 0; i < 9; ++i) c->cell[i] = cell[i] * c->kgrid[i / 3];
  for (int i = 0; i < 3; ++i) c->opts.fft[i] = c->opts.fft[i] > 0 ? c->opts.fft[i] * c->kgrid[i] : 0;
  std::vector<int> spec_all((size_t)natoms * nk);
  std::vector<double> pos_all((size_t)3 * natoms * nk);
  for (long long t = 0; t < nk; ++t) std::copy(species_of_atom, species_of_atom + natoms, spec_all.begin() + t * natoms);
  expand_positions(c->kgrid, cell, natoms, pos, pos_all.data());
  natoms = (int)(natoms * nk);
  nbands = (int)(nbands * nk);
  species_of_atom = spec_all.data();
  pos = pos_all.data();
  c->species.assign(sp, sp + nspecies);
  c->spec.assign(species_of_atom, species_of_atom + natoms);
  c->pos.assign(pos, pos + 3 * natoms);
  c->ecut = ecut;
  c->nb = nbands;
  c->precision = c->opts.precision ? 1 : 0;
  c->tsize = c->precision ? sizeof(float) : sizeof(double);
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    delete c;
    sgo::set_error("cudaGetDevice failed");
    return SGO_ERR_CUDA;
  }
  for (int s = 0; s < nspecies; ++s)
    if (!(sp[s].rp > 0.0) || (sp[s].d_p != 0.0 && !(sp[s].rp_p > 0.0)) || !std::isfinite(sp[s].d_p)) {
      delete c;
      sgo::set_error("projector widths must be positive (rp, and rp_p where d_p != 0)");
      return SGO_ERR_ARG;
    }
  double nel = 0.0;
  for (int a = 0; a < natoms; ++a) {
    if (species_of_atom[a] < 0 || species_of_atom[a] >= nspecies) {
      delete c;
      sgo::set_error("species index out of range");
      return SGO_ERR_ARG;
    }
    nel += sp[species_of_atom[a]].z_val;
  }
  const double need = c->opts.kT > 0.0 ? nel / 2.0 + 1.0 : nel / 2.0;
  if (nbands < (int)std::ceil(need - 1e-9) || (c->opts.kT <= 0.0 && std::fabs(nel / 2.0 - std::round(nel / 2.0)) > 1e-9)) {
    delete c;
    sgo::set_error("too few bands for the electrons (or odd electron count with integer occupations)");
    return SGO_ERR_ARG;
  }
  c->nb_int = nbands + (c->opts.extra_bands < 0 ? 4 + nbands / 32 : c->opts.extra_bands);
  if (c->opts.max_scf < 1 || c->opts.pulay_hist < 1 || c->opts.ncg < 1 || !(c->opts.eig_tol >= 0.0) ||
      c->opts.max_polish < 0 || !(c->opts.watchdog_ms >= 0.0)) {
    delete c;
    sgo::set_error("invalid SCF options");
    return SGO_ERR_ARG;
  }
  // geometry check through set_positions after set-up needs the device; check here first
  sgo_status s = sgo::ctx_setup(c);
  if (s == SGO_OK) s = sgo::set_positions(c, pos);
  if (s == SGO_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) s = SGO_ERR_CUDA;
  if (s != SGO_OK) {
    delete c;
    return s;
  }
  *out = c;
  return SGO_OK;
}

sgo_status sgo_scf(sgo_ctx* c, const double* pos, int* n_iter_out, double* resid_out) {
  if (!c) return SGO_ERR_ARG;
  if (pos) {
    sgo_status s = set_user_positions(c, pos);
    if (s != SGO_OK) return s;
  }
  std::unique_ptr<sgo::Engine> e(solo_engine(c));
  if (!e->ok()) return SGO_ERR_CUDA;
  sgo_status s = e->run(false, nullptr);
  if (n_iter_out) *n_iter_out = c->last_iter;
  if (resid_out) *resid_out = c->last_resid;
  return s;
}

sgo_status sgo_energy_forces(sgo_ctx* c, const double* pos, double* energy, double* forces) {
  if (!c) return SGO_ERR_ARG;
  if (pos) {
    sgo_status s = set_user_positions(c, pos);
    if (s != SGO_OK) return s;
  }
  std::unique_ptr<sgo::Engine> e(solo_engine(c));
  if (!e->ok()) return SGO_ERR_CUDA;
  sgo_status s = e->run(true, nullptr);
  if (energy) *energy = user_energy(c);
  if (forces) user_forces(c, forces);
  return s;
}

sgo_status sgo_batch_create(int n, sgo_ctx* const* ctxs, sgo_batch** out) {
  if (!out || n < 1 || !ctxs) return SGO_ERR_ARG;
  *out = nullptr;
  sgo_batch* b = new (std::nothrow) sgo_batch();
  if (!b) return SGO_ERR_OOM;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) {
      delete b;
      return SGO_ERR_ARG;
    }
    b->ctxs.push_back(ctxs[i]);
  }
  const sgo_opts& o = b->ctxs[0]->opts;
  for (int i = 1; i < n; ++i)
    if (b->ctxs[i]->precision != b->ctxs[0]->precision || b->ctxs[i]->opts.eigensolver != o.eigensolver ||
        b->ctxs[i]->opts.xc != o.xc) {
      sgo::set_error("the members of a batch must share precision, eigensolver and exchange-correlation");
      delete b;
      return SGO_ERR_ARG;
    }
  b->members = split_members(b->ctxs, sub_batch_count(n, o));
  std::vector<int> foff(n + 1, 0);
  for (int i = 0; i < n; ++i) foff[i + 1] = foff[i] + 3 * b->ctxs[i]->d.natom;
  for (const auto& m : b->members) {
    std::vector<sgo_ctx*> sub;
    std::vector<int> off;
    for (int i : m) {
      sub.push_back(b->ctxs[i]);
      off.push_back(foff[i]);
    }
    std::unique_ptr<sgo::Engine> e(new (std::nothrow) sgo::Engine(sub, b->ctxs[0]->stream));
    if (!e || !e->ok() || !e->set_slots(m, off)) {
      delete b;
      return SGO_ERR_CUDA;
    }
    e->enable_graphs(o.graph != 0);
    if (o.autotune) e->autotune();
    if (!e->ok()) {
      delete b;
      return SGO_ERR_CUDA;
    }
    b->engs.push_back(std::move(e));
  }
  if (cudaStreamSynchronize(b->ctxs[0]->stream) != cudaSuccess) {
    delete b;
    return SGO_ERR_CUDA;
  }
  *out = b;
  return SGO_OK;
}

sgo_status sgo_batch_tuning(const sgo_batch* b, int* knobs) {
  if (!b || !knobs) return SGO_ERR_ARG;
  b->engs[0]->tuning(knobs);
  return SGO_OK;
}

sgo_status sgo_energy_forces_batch(sgo_batch* b, const double* const* pos, double* energies, double* const* forces,
                                   sgo_status* per_item) {
  if (!b) return SGO_ERR_ARG;
  const int n = (int)b->ctxs.size();
  std::vector<sgo_status> st(n, SGO_OK);
  if (pos) {
    for (int i = 0; i < n; ++i) {
      if (!pos[i]) continue;
      sgo_status s = set_user_positions(b->ctxs[i], pos[i]);
      if (s == SGO_ERR_CUDA) return s;
      st[i] = s;
    }
  }
  std::vector<sgo_status> run_st(n, SGO_OK);
  if (run_batch(b, nullptr, &run_st) == SGO_ERR_CUDA) return SGO_ERR_CUDA;
  for (int i = 0; i < n; ++i) {
    sgo_ctx* c = b->ctxs[i];
    if (st[i] == SGO_OK) st[i] = run_st[i];
    if (energies) energies[i] = user_energy(c);
    if (forces && forces[i]) user_forces(c, forces[i]);
    if (per_item) per_item[i] = st[i];
  }
  return SGO_OK;
}

sgo_status sgo_energy_forces_batch_device(sgo_batch* b, const double* pos_dev, double* energies_dev,
                                          double* forces_dev, int* status_dev) {
  if (!b || !energies_dev || !forces_dev || !status_dev) return SGO_ERR_ARG;
  for (auto* c : b->ctxs)
    if (c->nk != 1) {
      sgo::set_error("a k-point member: the device-array batch call takes Gamma-point members only");
      return SGO_ERR_ARG;
    }
  const sgo::Engine::DeviceIO io{pos_dev, energies_dev, forces_dev, status_dev};
  return run_batch(b, &io, nullptr);
}

sgo_status sgo_relax_batch(sgo_batch* b, sgo_relax* const* relax, int max_rounds, int* rounds,
                           sgo_status* per_item) {
  if (rounds) *rounds = 0;
  if (!b || !relax || max_rounds < 0) return SGO_ERR_ARG;
  const int n = (int)b->ctxs.size();
  for (int i = 0; i < n; ++i)
    if (!relax[i] || sgo_relax_natoms(relax[i]) != b->ctxs[i]->nat_user) return SGO_ERR_ARG;
  std::vector<std::vector<double>> pos(n), F(n);
  std::vector<const double*> pp(n);
  std::vector<double*> fp(n);
  std::vector<double> E(n);
  std::vector<sgo_status> st(n, SGO_OK), evs(n);
  std::vector<int> state(n, 0);
  for (int i = 0; i < n; ++i) {
    pos[i].resize(3 * b->ctxs[i]->nat_user);
    F[i].resize(pos[i].size());
    sgo_relax_positions(relax[i], pos[i].data());
    sgo_relax_info(relax[i], nullptr, &state[i]);
    pp[i] = pos[i].data();
    fp[i] = F[i].data();
  }
  int r = 0;
  for (; r < max_rounds; ++r) {
    bool any = false;
    for (int i = 0; i < n; ++i) any = any || (state[i] == 0 && st[i] == SGO_OK);
    if (!any) break;
    const sgo_status s = sgo_energy_forces_batch(b, pp.data(), E.data(), fp.data(), evs.data());
    if (s != SGO_OK) return s;
    for (int i = 0; i < n; ++i) b->ctxs[i]->warm = true;  // the next relaxation round starts from these states
    // the drivers are independent: step them on all host cores
    std::atomic<int> next(0);
    auto work = [&]() {
      for (int i = next++; i < n; i = next++) {
        if (state[i] != 0 || st[i] != SGO_OK) continue;
        if (evs[i] != SGO_OK) {
          st[i] = evs[i];
          continue;
        }
        const sgo_status rs = sgo_relax_step(relax[i], E[i], F[i].data(), pos[i].data(), &state[i]);
        if (rs != SGO_OK) st[i] = rs;
      }
    };
    const int nt = std::max(1, std::min(n, (int)std::thread::hardware_concurrency()));
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) pool.emplace_back(work);
    work();
    for (auto& t : pool) t.join();
  }
  if (rounds) *rounds = r;
  if (per_item)
    for (int i = 0; i < n; ++i) per_item[i] = st[i];
  return SGO_OK;
}

sgo_status sgo_de_generation(sgo_batch* b, const double cell[9], const int* species, double* pop, double* f,
                             const double* u, int scheme, double d_min, const sgo_relax_opts* ro, int max_rounds,
                             int* replaced, double* child_f) {
  if (!b || !cell || !species || !pop || !f || !u || max_rounds < 0) return SGO_ERR_ARG;
  const int np = (int)b->ctxs.size();
  const int na = b->ctxs[0]->nat_user;
  for (auto* c : b->ctxs)
    if (c->nat_user != na) return SGO_ERR_ARG;
  const size_t sz = 3 * (size_t)na;
  std::vector<double> kids(sz * np);
  sgo_status s = sgo_de_offspring(np, na, cell, species, pop, f, u, scheme, d_min, kids.data());
  if (s != SGO_OK) return s;
  std::vector<sgo_relax*> drv(np, nullptr);
  auto cleanup = [&]() {
    for (auto* d : drv) sgo_relax_destroy(d);
  };
  for (int i = 0; i < np; ++i) {
    s = sgo_relax_create(na, cell, kids.data() + sz * i, ro, &drv[i]);
    if (s != SGO_OK) {
      cleanup();
      return s;
    }
    b->ctxs[i]->warm = false;  // a new structure: the first evaluation starts from the atomic guess
  }
  std::vector<sgo_status> st(np, SGO_OK);
  int rounds = 0;
  s = sgo_relax_batch(b, drv.data(), max_rounds, &rounds, st.data());
  if (s != SGO_OK) {
    cleanup();
    return s;
  }
  std::vector<double> best(sz);
  for (int i = 0; i < np; ++i) {
    double e = INFINITY;
    const bool ok = st[i] == SGO_OK && sgo_relax_best(drv[i], &e, best.data()) == SGO_OK;
    if (!ok) e = INFINITY;
    if (child_f) child_f[i] = e;
    const bool better = ok && e < f[i];
    if (better) {
      std::memcpy(pop + sz * i, best.data(), sizeof(double) * sz);
      f[i] = e;
    }
    if (replaced) replaced[i] = better ? 1 : 0;
  }
  cleanup();
  return SGO_OK;
}

sgo_status sgo_batch_timer(sgo_batch* b, const char* kernel) {
  if (!b) return SGO_ERR_ARG;
  for (auto& e : b->engs)
    if (!e->timer_select(kernel)) {
      sgo::set_error("unknown kernel class");
      return SGO_ERR_ARG;
    }
  return SGO_OK;
}

sgo_status sgo_batch_timer_read(sgo_batch* b, double out[4]) {
  if (!b || !out) return SGO_ERR_ARG;
  // sums over the sub-batches (the timed mode runs them one after another)
  for (int i = 0; i < 4; ++i) out[i] = 0.0;
  for (auto& e : b->engs) {
    double v[4];
    int launches = 0;
    e->timer_read(&v[0], &launches, &v[2], &v[3]);
    out[0] += v[0];
    out[1] += launches;
    out[2] += v[2];
    out[3] += v[3];
  }
  return SGO_OK;
}

sgo_status sgo_batch_launches(sgo_batch* b, long long* count) {
  if (!b || !count) return SGO_ERR_ARG;
  *count = 0;
  for (auto& e : b->engs) *count += e->take_launches();
  return SGO_OK;
}

sgo_status sgo_get_eigen(sgo_ctx* c, double* eig, double* occ) {
  if (!c) return SGO_ERR_ARG;
  if (eig) std::memcpy(eig, c->h_eps.data(), sizeof(double) * c->nb);
  if (occ) std::memcpy(occ, c->h_occ.data(), sizeof(double) * c->nb);
  return SGO_OK;
}

sgo_status sgo_get_terms(sgo_ctx* c, double terms[8]) {
  if (!c || !terms) return SGO_ERR_ARG;
  const double* s = c->h_scal.data();
  terms[0] = s[sgo::SC_EKIN];
  terms[1] = s[sgo::SC_ENL];
  terms[2] = s[sgo::SC_ELOC];
  terms[3] = s[sgo::SC_EH];
  terms[4] = s[sgo::SC_EXC];
  terms[5] = s[sgo::SC_EEW];
  terms[6] = s[sgo::SC_MTS];
  terms[7] = s[sgo::SC_FREE];
  for (int i = 0; i < 8; ++i) terms[i] /= c->nk;  // (per cell of the caller)
  return SGO_OK;
}

sgo_status sgo_get_info(sgo_ctx* c, int info[10]) {
  if (!c || !info) return SGO_ERR_ARG;
  info[0] = c->d.npw;
  info[1] = c->d.nhalf;
  info[2] = c->d.ncp;
  info[3] = c->d.n1;
  info[4] = c->d.n2;
  info[5] = c->d.n3;
  info[6] = c->nb;
  info[7] = c->nat_user;
  info[8] = c->last_iter;
  info[9] = c->precision;
  return SGO_OK;
}

sgo_status sgo_get_stats(sgo_ctx* c, double stats[8]) {
  if (!c || !stats) return SGO_ERR_ARG;
  stats[0] = c->last_iter;
  stats[1] = c->h_scal[sgo::SC_RRSWEEPS];
  stats[2] = c->h_scal[sgo::SC_RESID];
  stats[3] = c->h_scal[sgo::SC_DF];
  stats[4] = c->h_scal[sgo::SC_POLISH];
  stats[5] = c->h_scal[sgo::SC_EIGRES];
  stats[6] = c->h_scal[sgo::SC_RRCAP];
  stats[7] = c->last_warm ? 1.0 : 0.0;
  return SGO_OK;
}

sgo_status sgo_get_state(sgo_ctx* c, double* rho_g, double* psi) {
  if (!c || (!rho_g && !psi)) return SGO_ERR_ARG;
  if (!c->have_state) {
    sgo::set_error("no state yet: run an evaluation or sgo_set_state first");
    return SGO_ERR_ARG;
  }
  std::unique_ptr<sgo::Engine> e(solo_engine(c));
  if (!e->ok()) return SGO_ERR_CUDA;
  return e->export_state(rho_g, psi);
}

sgo_status sgo_set_state(sgo_ctx* c, const double* rho_g, const double* psi) {
  if (!c || !rho_g || !psi) return SGO_ERR_ARG;
  const size_t ng = (size_t)c->d.ngrid, np = (size_t)c->nb * c->d.npw;
  for (size_t i = 0; i < 2 * ng; ++i)
    if (!std::isfinite(rho_g[i])) {
      sgo::set_error("non-finite density in the imported state");
      return SGO_ERR_ARG;
    }
  for (size_t i = 0; i < np; ++i)
    if (!std::isfinite(psi[i])) {
      sgo::set_error("non-finite wavefunction in the imported state");
      return SGO_ERR_ARG;
    }
  std::unique_ptr<sgo::Engine> e(solo_engine(c));
  if (!e->ok()) return SGO_ERR_CUDA;
  const sgo_status s = e->import_state(rho_g, psi);
  if (s == SGO_OK) {
    c->have_state = true;
    c->warm = true;
  }
  return s;
}

sgo_status sgo_get_basis(sgo_ctx* c, int* miller) {
  if (!c || !miller) return SGO_ERR_ARG;
  const int nh = c->d.nhalf;
  std::vector<int> m(3 * (size_t)nh);
  if (nh > 0 && cudaMemcpy(m.data(), c->d.ent_m, sizeof(int) * 3 * nh, cudaMemcpyDeviceToHost) != cudaSuccess)
    return SGO_ERR_CUDA;
  miller[0] = miller[1] = miller[2] = 0;
  for (int e = 0; e < nh; ++e) {
    miller[3 * (e + 1) + 0] = m[e];
    miller[3 * (e + 1) + 1] = m[nh + e];
    miller[3 * (e + 1) + 2] = m[2 * nh + e];
  }
  return SGO_OK;
}

sgo_status sgo_get_density(sgo_ctx* c, double* rho) {
  if (!c || !rho) return SGO_ERR_ARG;
  std::unique_ptr<sgo::Engine> e(solo_engine(c));
  if (!e->ok()) return SGO_ERR_CUDA;
  return e->export_density(rho);
}

sgo_status sgo_grid_fft(sgo_ctx* c, int sign, const double* in, double* out) {
  if (!c || !in || !out || (sign != 1 && sign != -1)) return SGO_ERR_ARG;
  std::unique_ptr<sgo::Engine> e(solo_engine(c));
  if (!e->ok()) return SGO_ERR_CUDA;
  return e->grid_transform(sign, in, out);
}

sgo_status sgo_apply_hamiltonian(sgo_ctx* c, const double* veff, int nvec, const double* psi, double* hpsi) {
  if (!c || !veff || !psi || !hpsi || nvec < 1 || nvec > c->nb) return SGO_ERR_ARG;
  std::unique_ptr<sgo::Engine> e(solo_engine(c));
  if (!e->ok()) return SGO_ERR_CUDA;
  return e->apply_h(veff, nvec, psi, hpsi);
}

sgo_status sgo_subspace_matrix(sgo_ctx* c, int nvec, const double* x, const double* y, double* out) {
  if (!c || !x || !y || !out || nvec < 1 || nvec > c->nb) return SGO_ERR_ARG;
  std::unique_ptr<sgo::Engine> e(solo_engine(c));
  if (!e->ok()) return SGO_ERR_CUDA;
  return e->subspace(nvec, x, y, out);
}

sgo_status sgo_block_update(sgo_ctx* c, int nvec, const double* x, const double* m, double alpha, double beta,
                            double* y) {
  if (!c || !x || !m || !y || nvec < 1 || nvec > c->nb) return SGO_ERR_ARG;
  std::unique_ptr<sgo::Engine> e(solo_engine(c));
  if (!e->ok()) return SGO_ERR_CUDA;
  return e->block_update(nvec, x, m, alpha, beta, y);
}

sgo_status sgo_density(sgo_ctx* c, int nvec, const double* psi, const double* occ, double* rho) {
  if (!c || !psi || !occ || !rho || nvec < 1 || nvec > c->nb) return SGO_ERR_ARG;
  std::unique_ptr<sgo::Engine> e(solo_engine(c));
  if (!e->ok()) return SGO_ERR_CUDA;
  return e->density(nvec, psi, occ, rho);
}

sgo_status sgo_set_warm(sgo_ctx* c, int on) {
  if (!c) return SGO_ERR_ARG;
  c->warm = on != 0;
  return SGO_OK;
}

void sgo_batch_destroy(sgo_batch* b) { delete b; }
void sgo_destroy(sgo_ctx* c) { delete c; }

const char* sgo_status_string(sgo_status s) {
  switch (s) {
    case SGO_OK: return "ok";
    case SGO_ERR_ARG: return "invalid argument";
    case SGO_ERR_GEOMETRY: return "invalid geometry";
    case SGO_ERR_CUDA: return "CUDA error";
    case SGO_ERR_OOM: return "out of device memory";
    case SGO_ERR_NOT_CONVERGED: return "SCF not converged";
    case SGO_ERR_TIMEOUT: return "device wait timed out";
    case SGO_ERR_NAN: return "non-finite result";
  }
  return "unknown status";
}

const char* sgo_last_error(void) { return sgo::last_error(); }

}  // extern "C"
