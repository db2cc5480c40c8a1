/*
 * des.c -- CPU oracle of the discrete-event simulation of the spatial hypercube
 * queue's loss system with general service times (the check of Section 5.5 of arXiv
 * 2603.03019, "Results for General Service Time Distributions", and its Table of MRT
 * and utilisation errors).
 *
 * TEST INFRASTRUCTURE ONLY, like hq_oracle.c: the tests, the smoke check and the
 * CPU-baseline leg of the benchmark use it; it shares no code with the CUDA library.
 *
 * The system (Section 2.1 with the zero-queue rule): calls arrive as a Poisson process
 * of rate lambda = sum_j lambda_j; a call comes from node j with probability
 * lambda_j / lambda and goes to the first idle unit of node j's preference list; if
 * every unit is busy it is lost.  Unit i's service times are i.i.d. with mean 1/nu_i
 * and one of five shapes (Section 5.5 sets every distribution's mean to 1/nu_i):
 *   0 exponential;
 *   1 log-normal with the exponential's variance (sigma^2 = ln 2, mu = ln m - ln2/2);
 *   2 gamma with scale 1/(5 nu_i) (shape 5: smaller variance), as the sum of 5
 *     exponentials of mean m/5;
 *   3 gamma with scale 1/(0.5 nu_i) (shape 1/2: larger variance), as m Z^2 with Z
 *     standard normal;
 *   4 uniform on [0, 2m] (smaller variance).
 * Normals by the Box-Muller transform.  Each replication starts empty at time 0; the
 * first `warmup` arrivals are not counted; the window runs from the arrival time of
 * call `warmup` to that of the last call.  Per replication and unit: the busy time in
 * the window (exact overlap of every service with the window), the calls served; per
 * replication: calls lost, the window length and the sum of the travel times
 * travel[j*N + i] of the served calls (the response time of Section 5.5's MRT, on
 * travel times the caller supplies).
 *
 * Random numbers: one counter-based generator, so that every replication and draw has
 * its own value regardless of how replications are scheduled: the splitmix64
 * finaliser (Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014) applied to key_r + (c + 1) * gamma, gamma = 0x9e3779b97f4a7c15, with
 * key_r = finaliser(seed + (r + 1) * gamma); draw c of arrival a is c = 8 a + k:
 * k = 0 inter-arrival time, 1 node, 2.. service time.  A uniform u in (0, 1] is
 * ((x >> 11) + 1) 2^-53.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define DES_GAMMA 0x9e3779b97f4a7c15ULL

static uint64_t des_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

static double des_u(uint64_t key, uint64_t c) {
  const uint64_t x = des_mix(key + (c + 1) * DES_GAMMA);
  return (double)((x >> 11) + 1) * 0x1.0p-53;
}

/* one standard normal from two uniforms (Box-Muller, cosine branch) */
static double des_normal(double u1, double u2) {
  const double two_pi = 6.283185307179586476925286766559;
  return sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
}

double or_des_service(int kind, double m, uint64_t key, uint64_t c0) {
  const double u2 = des_u(key, c0), u3 = des_u(key, c0 + 1);
  switch (kind) {
    case 0:
      return -m * log(u2);
    case 1: {
      const double s2 = log(2.0);
      const double mu = log(m) - 0.5 * s2;
      return exp(mu + sqrt(s2) * des_normal(u2, u3));
    }
    case 2: {
      const double prod = u2 * u3 * des_u(key, c0 + 2) * des_u(key, c0 + 3) * des_u(key, c0 + 4);
      return -(m / 5.0) * log(prod);
    }
    case 3: {
      const double z = des_normal(u2, u3);
      return m * (z * z);
    }
    case 4:
      return (2.0 * m) * u2;
    default:
      return -1.0;
  }
}

double or_des_uniform(uint64_t seed, int64_t r, uint64_t c) {
  return des_u(des_mix(seed + (uint64_t)(r + 1) * DES_GAMMA), c);
}

/* Returns 0, or -1 for bad arguments. */
int or_des_loss(int N, int J, const double* lam_j, const double* nu, const int32_t* pref,
                const double* travel, int kind, int64_t reps, int64_t arrivals, int64_t warmup,
                uint64_t seed, double* busy, int64_t* served, int64_t* lost, double* window,
                double* resp) {
  if (N < 1 || N > 64 || J < 1 || reps < 1 || arrivals < 2 || warmup < 0 || warmup >= arrivals - 1 ||
      kind < 0 || kind > 4)
    return -1;
  double* cdf = (double*)malloc(sizeof(double) * (size_t)J);
  double* fr = (double*)malloc(sizeof(double) * (size_t)N);
  if (!cdf || !fr) {
    free(cdf);
    free(fr);
    return -1;
  }
  double acc = 0.0;
  for (int j = 0; j < J; j++) {
    acc += lam_j[j];
    cdf[j] = acc;
  }
  const double lam = acc;
  for (int64_t r = 0; r < reps; r++) {
    const uint64_t key = des_mix(seed + (uint64_t)(r + 1) * DES_GAMMA);
    for (int i = 0; i < N; i++) {
      fr[i] = 0.0;
      busy[r * N + i] = 0.0;
      served[r * N + i] = 0;
    }
    lost[r] = 0;
    resp[r] = 0.0;
    double t = 0.0, t0 = 0.0;
    for (int64_t a = 0; a < arrivals; a++) {
      const uint64_t c = 8 * (uint64_t)a;
      t = t + (-log(des_u(key, c)) / lam);
      const int in_window = a >= warmup;
      if (a == warmup) {
        /* the window opens: services in progress count from here */
        t0 = t;
        for (int i = 0; i < N; i++)
          if (fr[i] > t0) busy[r * N + i] = fr[i] - t0;
      }
      /* node: the first j whose cumulative rate reaches u lambda */
      const double target = des_u(key, c + 1) * lam;
      int lo = 0, hi = J - 1;
      while (lo < hi) {
        const int mid = (lo + hi) / 2;
        if (cdf[mid] >= target) hi = mid;
        else lo = mid + 1;
      }
      const int j = lo;
      int unit = -1;
      for (int h = 0; h < N; h++) {
        const int i = pref[(int64_t)j * N + h];
        if (fr[i] <= t) {
          unit = i;
          break;
        }
      }
      if (unit < 0) {
        if (in_window) lost[r]++;
        continue;
      }
      const double s = or_des_service(kind, 1.0 / nu[unit], key, c + 2);
      fr[unit] = t + s;
      if (in_window) {
        busy[r * N + unit] += s;
        served[r * N + unit]++;
        resp[r] += travel[(int64_t)j * N + unit];
      }
    }
    /* the window closes at the last arrival: cut every unit's last service there */
    for (int i = 0; i < N; i++)
      if (fr[i] > t) busy[r * N + i] -= fr[i] - t;
    window[r] = t - t0;
  }
  free(cdf);
  free(fr);
  return 0;
}
