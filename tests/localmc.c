/*
 * localmc.c -- textbook local Monte Carlo of hard disks (Metropolis
 * displacement moves), the reference the paper compares its event-chain
 * variants against in Fig. 3.  TEST INFRASTRUCTURE: an independent sampler
 * of the uniform measure on non-overlapping configurations, sharing no code
 * and no random stream with the oracle.
 *
 * One sweep is N moves: a disk drawn uniformly is displaced by a vector
 * uniform on [-delta, delta]^2 and the move is accepted unless the disk then
 * overlaps another (minimum-image distance < sigma).  Random numbers come
 * from splitmix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014).  After each sweep the ordered-pair counts of
 * the minimum-image distances in [r0, r0 + nb dr) are accumulated.
 */
#include <math.h>
#include <stdint.h>

static uint64_t splitmix64(uint64_t* s) {
  uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static double unif(uint64_t* s) { return (double)(splitmix64(s) >> 11) * 0x1.0p-53; }

static double wrapc(double v, double L) {
  v -= L * floor(v / L + 0.5);
  return v;
}

/* Returns the number of accepted moves. */
long long localmc_run(int N, double L, double sigma, double delta, double* x, double* y,
                      long long sweeps, uint64_t seed, double r0, double dr, int nb,
                      long long* counts) {
  uint64_t s = seed;
  const double s2 = sigma * sigma;
  long long acc = 0;
  for (long long sw = 0; sw < sweeps; ++sw) {
    for (int mv = 0; mv < N; ++mv) {
      const int i = (int)(unif(&s) * N);
      double nx = x[i] + (2.0 * unif(&s) - 1.0) * delta;
      double ny = y[i] + (2.0 * unif(&s) - 1.0) * delta;
      nx -= L * floor(nx / L);
      ny -= L * floor(ny / L);
      int ok = 1;
      for (int j = 0; j < N && ok; ++j) {
        if (j == i) continue;
        const double dx = wrapc(nx - x[j], L), dy = wrapc(ny - y[j], L);
        if (dx * dx + dy * dy < s2) ok = 0;
      }
      if (ok) {
        x[i] = nx;
        y[i] = ny;
        acc++;
      }
    }
    if (counts) {
      for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
          if (j == i) continue;
          const double dx = wrapc(x[j] - x[i], L), dy = wrapc(y[j] - y[i], L);
          const double d = sqrt(dx * dx + dy * dy);
          const int b = (int)floor((d - r0) / dr);
          if (b >= 0 && b < nb) counts[b]++;
        }
    }
  }
  return acc;
}

/* The same in three dimensions (spheres of diameter sigma in a periodic
 * cube; displacements uniform on [-delta, delta]^3). */
long long localmc3_run(int N, double L, double sigma, double delta, double* x, double* y,
                       double* z, long long sweeps, uint64_t seed, double r0, double dr, int nb,
                       long long* counts) {
  uint64_t s = seed;
  const double s2 = sigma * sigma;
  long long acc = 0;
  for (long long sw = 0; sw < sweeps; ++sw) {
    for (int mv = 0; mv < N; ++mv) {
      const int i = (int)(unif(&s) * N);
      double nx = x[i] + (2.0 * unif(&s) - 1.0) * delta;
      double ny = y[i] + (2.0 * unif(&s) - 1.0) * delta;
      double nz = z[i] + (2.0 * unif(&s) - 1.0) * delta;
      nx -= L * floor(nx / L);
      ny -= L * floor(ny / L);
      nz -= L * floor(nz / L);
      int ok = 1;
      for (int j = 0; j < N && ok; ++j) {
        if (j == i) continue;
        const double dx = wrapc(nx - x[j], L), dy = wrapc(ny - y[j], L), dz = wrapc(nz - z[j], L);
        if (dx * dx + dy * dy + dz * dz < s2) ok = 0;
      }
      if (ok) {
        x[i] = nx;
        y[i] = ny;
        z[i] = nz;
        acc++;
      }
    }
    if (counts) {
      for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
          if (j == i) continue;
          const double dx = wrapc(x[j] - x[i], L), dy = wrapc(y[j] - y[i], L),
                       dz = wrapc(z[j] - z[i], L);
          const double d = sqrt(dx * dx + dy * dy + dz * dz);
          const int b = (int)floor((d - r0) / dr);
          if (b >= 0 && b < nb) counts[b]++;
        }
    }
  }
  return acc;
}
