// ecmc_tune.cu -- the degree of parallelisation, chosen by measurement
// (Sec. 4: eqs. nm, lambda0 and criterion, Figs. 5-6).
//
// ecmc_tune_geometry runs one trial per candidate (cells per side, ell), with
// n_m from eq. (nm), from the caller's configuration (or the square lattice):
// warm-up sweeps, then sweeps timed with CUDA events on a stream of its own
// until at least min_seconds have passed.  Per trial it records events/s,
// sweeps/s, the mean free path lambda0 the chains actually saw (displacement
// over contacts + walls + chain ends), the criterion's displacement
// ell* = L lambda0 / (sqrt(n) sigma) with that lambda0, and a sampling proxy:
//   ECMC_TUNE_EVENTS  events per second;
//   ECMC_TUNE_MSD     mean square displacement per disk per sweep, times
//                     sweeps per second: how fast the disks move in wall
//                     time (displacements accumulated sweep by sweep by the
//                     minimum image, so wraps do not count);
//   ECMC_TUNE_TAU     sweeps per second over the autocorrelation time of the
//                     hexatic order parameter in sweeps (eq. tau, Psi after
//                     every sweep of the trial): decorrelation per wall time,
//                     the quantity Fig. 6 compares.
// The trial with the largest score is the choice.  Every trial is a
// separate handle built through the public entry points, so the tuning
// leaves the caller's system untouched.
#include <cmath>
#include <cstring>
#include <vector>

#include "ecmc.h"
#include "ecmc_device.cuh"
#include "ecmc_internal.cuh"

namespace {

__global__ void k_accum_disp(const double* __restrict__ prev, const double* __restrict__ cur,
                             int64_t n2, double L, double* __restrict__ disp) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n2) disp[i] += ecmc::wrap_half(cur[i] - prev[i], L);
}

struct Scratch {
  double *prev = nullptr, *cur = nullptr, *disp = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  ~Scratch() {
    cudaFree(prev);
    cudaFree(cur);
    cudaFree(disp);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (s) cudaStreamDestroy(s);
  }
};

int run_trial(const ecmc_replica_desc_t& desc, const double* xy, int warm, int trial,
              double min_seconds, int proxy, Scratch& sc, ecmc_geom_trial_t* t) {
  ecmc_t h = nullptr;
  int rc = ecmc_create_batch(&h, &desc, 1);
  if (rc) return rc;
  struct Closer {
    ecmc_t h;
    ~Closer() { ecmc_destroy(h); }
  } closer{h};
  if ((rc = ecmc_set_stream(h, sc.s))) return rc;
  if (xy && (rc = ecmc_set_positions(h, xy, 0, 0))) return rc;
  ecmc_replica_desc_t used;
  if ((rc = ecmc_replica_desc(h, 0, &used))) return rc;
  t->n_m = used.n_m;
  if ((rc = ecmc_sweep(h, warm)) || (rc = ecmc_synchronize(h)) || (rc = ecmc_reset_stats(h)))
    return rc;
  // timed sweeps, in batches of `trial`, until min_seconds have passed
  int64_t swept = 0;
  float ms = 0.0f;
  if (cudaEventRecord(sc.a, sc.s) != cudaSuccess) return ECMC_ERR_CUDA;
  for (;;) {
    if ((rc = ecmc_sweep(h, trial))) return rc;
    swept += trial;
    if (cudaEventRecord(sc.b, sc.s) != cudaSuccess || cudaEventSynchronize(sc.b) != cudaSuccess ||
        cudaEventElapsedTime(&ms, sc.a, sc.b) != cudaSuccess)
      return ECMC_ERR_CUDA;
    if (ms * 1e-3 >= min_seconds) break;
  }
  ecmc_counters_t c;
  if ((rc = ecmc_counters(h, &c))) return rc;
  const double sec = ms * 1e-3;
  t->ms_per_sweep = ms / (double)swept;
  t->sweeps = swept;
  t->events_per_s = (double)c.events / sec;
  t->sweeps_per_s = (double)swept / sec;
  const double legs = (double)(c.events + c.wall_hits + c.chains);
  t->lambda0 = legs > 0.0 ? c.sum_disp / legs : 0.0;
  const double n_blocks = (double)desc.cells_x * (double)desc.cells_y / 4.0;
  t->ell_star = desc.L * t->lambda0 / (std::sqrt(n_blocks) * desc.sigma);
  t->msd_per_sweep = 0.0;
  t->tau_sweeps = 0.0;
  const int64_t N = desc.N;
  if (proxy == ECMC_TUNE_MSD) {
    const size_t bytes = sizeof(double) * 2 * (size_t)N;
    if ((rc = ecmc_positions(h, sc.prev, 1))) return rc;
    if (cudaMemsetAsync(sc.disp, 0, bytes, sc.s) != cudaSuccess) return ECMC_ERR_CUDA;
    for (int i = 0; i < trial; ++i) {
      if ((rc = ecmc_sweep(h, 1)) || (rc = ecmc_positions(h, sc.cur, 1))) return rc;
      k_accum_disp<<<(unsigned)((2 * N + 255) / 256), 256, 0, sc.s>>>(sc.prev, sc.cur, 2 * N,
                                                                        desc.L, sc.disp);
      if (cudaGetLastError() != cudaSuccess) return ECMC_ERR_CUDA;
      std::swap(sc.prev, sc.cur);
    }
    std::vector<double> d(2 * (size_t)N);
    if (cudaMemcpyAsync(d.data(), sc.disp, bytes, cudaMemcpyDeviceToHost, sc.s) != cudaSuccess ||
        cudaStreamSynchronize(sc.s) != cudaSuccess)
      return ECMC_ERR_CUDA;
    double sum = 0.0;
    for (int64_t i = 0; i < N; ++i) sum += d[2 * i] * d[2 * i] + d[2 * i + 1] * d[2 * i + 1];
    t->msd_per_sweep = sum / (double)N / (double)trial;
    t->score = t->msd_per_sweep * t->sweeps_per_s;
  } else if (proxy == ECMC_TUNE_TAU) {
    std::vector<double> series(2 * (size_t)trial);
    for (int i = 0; i < trial; ++i) {
      if ((rc = ecmc_sweep(h, 1)) || (rc = ecmc_hexatic(h, 0.0, &series[2 * i], nullptr,
                                                         nullptr, nullptr)))
        return rc;
    }
    double tau = 0.0;
    if ((rc = ecmc_autocorrelation_time(series.data(), trial, 1, trial / 4 > 1 ? trial / 4 : 1, &tau,
                                        nullptr)))
      return rc;
    t->tau_sweeps = tau;
    t->score = (std::isfinite(tau) && tau > 0.0) ? t->sweeps_per_s / tau : 0.0;
  } else {
    t->score = t->events_per_s;
  }
  return ECMC_OK;
}

}  // namespace

extern "C" int ecmc_tune_geometry(const ecmc_replica_desc_t* base, const double* xy,
                                  const int* cells, int n_cells, const double* ells, int n_ells,
                                  int warm_sweeps, int trial_sweeps, double min_seconds,
                                  int proxy, ecmc_geom_trial_t* trials, int* best) {
  if (!base || !cells || !ells || !trials || !best || n_cells < 1 || n_ells < 1 ||
      warm_sweeps < 0 || trial_sweeps < 1 || !(min_seconds >= 0.0) ||
      (proxy != ECMC_TUNE_EVENTS && proxy != ECMC_TUNE_MSD && proxy != ECMC_TUNE_TAU))
    return ecmc::report_error(ECMC_ERR_ARG, "bad tuning arguments");
  if (proxy == ECMC_TUNE_TAU && trial_sweeps < 8)
    return ecmc::report_error(ECMC_ERR_ARG, "the tau proxy needs at least 8 sweeps per trial");
  Scratch sc;
  const size_t bytes = sizeof(double) * 2 * (size_t)base->N;
  if (cudaStreamCreateWithFlags(&sc.s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&sc.a) != cudaSuccess || cudaEventCreate(&sc.b) != cudaSuccess)
    return ecmc::report_error(ECMC_ERR_CUDA, "stream or event creation failed");
  if (proxy == ECMC_TUNE_MSD &&
      (cudaMalloc(&sc.prev, bytes) != cudaSuccess || cudaMalloc(&sc.cur, bytes) != cudaSuccess ||
       cudaMalloc(&sc.disp, bytes) != cudaSuccess)) {
    cudaGetLastError();
    return ecmc::report_error(ECMC_ERR_OOM, "tuning scratch allocation failed");
  }
  *best = -1;
  double best_score = -1.0;
  int k = 0;
  for (int ic = 0; ic < n_cells; ++ic) {
    for (int ie = 0; ie < n_ells; ++ie, ++k) {
      ecmc_geom_trial_t* t = &trials[k];
      std::memset(t, 0, sizeof(*t));
      t->cells = cells[ic];
      t->ell = ells[ie];
      t->score = -1.0;
      ecmc_replica_desc_t d = *base;
      d.cells_x = d.cells_y = cells[ic];
      d.ell = ells[ie];
      d.n_m = 0;  // eq. (nm)
      // cells of side above 2 sigma (the frame of a cell spans w + 2 sigma)
      if (cells[ic] < 2 || (cells[ic] & 1) || !(base->L / cells[ic] > 2.0 * base->sigma) ||
          !(ells[ie] > 0.0)) {
        t->status = ECMC_ERR_ARG;
        continue;
      }
      t->status = run_trial(d, xy, warm_sweeps, trial_sweeps, min_seconds, proxy, sc, t);
      if (t->status != ECMC_OK) {
        t->score = -1.0;
        if (t->status == ECMC_ERR_CUDA) return t->status;
        continue;
      }
      if (t->score > best_score) {
        best_score = t->score;
        *best = k;
      }
    }
  }
  if (*best < 0) return ecmc::report_error(ECMC_ERR_ARG, "no candidate could run");
  return ECMC_OK;
}
