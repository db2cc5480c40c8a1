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
 * k = 0 inter-arrival time, 1 node, 2.. service time.  The node's uniform is
 * ((x >> 11) + 1) 2^-53 in (0, 1]; the variates' uniforms are ((x >> 40) + 1) 2^-24,
 * exact in FP32.
 *
 * Precision: the variates (inter-arrival and service times) are formed in FP32 -- their
 * relative rounding, about 1e-7, is far below any statistical effect -- with the
 * logarithm, exponential and cosine written here from their series (below), one IEEE
 * operation per step (the library's simulation does the same steps, so both take the
 * same decisions); the clock, busy times and response sums accumulate in FP64.
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

static double des_u53(uint64_t key, uint64_t c) {
  const uint64_t x = des_mix(key + (c + 1) * DES_GAMMA);
  return (double)((x >> 11) + 1) * 0x1.0p-53;
}

static float des_u24(uint64_t key, uint64_t c) {
  const uint64_t x = des_mix(key + (c + 1) * DES_GAMMA);
  return (float)((x >> 40) + 1) * 0x1.0p-24f;
}

/* ---- FP32 elementary functions from their series --------------------------------- */

/* ln x for a positive normal x: x = m 2^e with m in [sqrt(1/2), sqrt(2)), then
 * ln m = 2 atanh(s) = 2 (s + s^3/3 + s^5/5 + s^7/7 + s^9/9), s = (m - 1)/(m + 1), |s| <= 0.172 */
float or_des_ln(float x) {
  uint32_t b;
  memcpy(&b, &x, 4);
  int e = (int)((b >> 23) & 0xffu) - 127;
  const uint32_t mb = (b & 0x7fffffu) | 0x3f800000u;
  float m;
  memcpy(&m, &mb, 4);
  if (m > 0x1.6a09e6p+0f) {
    m = m * 0.5f;
    e += 1;
  }
  const float s = (m - 1.0f) / (m + 1.0f);
  const float z = s * s;
  float q = 0x1.c71c72p-4f;     /* 1/9 */
  q = q * z + 0x1.24924ap-3f;   /* 1/7 */
  q = q * z + 0x1.99999ap-3f;   /* 1/5 */
  q = q * z + 0x1.555556p-2f;   /* 1/3 */
  q = q * z + 1.0f;
  const float lnm = (s + s) * q;
  const float ef = (float)e;
  /* ln 2 = hi + lo with hi of 16 bits, so ef hi is exact (Cody and Waite's split) */
  const float lo = ef * 0x1.7f7d1cp-20f + lnm;
  return ef * 0x1.62e4p-1f + lo;
}

/* e^y for |y| < 80: y = k ln2 + r, |r| <= ln2/2, e^r from its Taylor series to r^8/8! */
float or_des_exp(float y) {
  const float k = floorf(y * 0x1.715476p+0f + 0.5f);
  float r = y - k * 0x1.62e4p-1f;   /* exact: k hi has at most 24 bits for |k| < 256 */
  r = r - k * 0x1.7f7d1cp-20f;
  float p = 0x1.a01a02p-16f;    /* 1/8! */
  p = p * r + 0x1.a01a02p-13f;  /* 1/7! */
  p = p * r + 0x1.6c16c2p-10f;  /* 1/6! */
  p = p * r + 0x1.111112p-7f;   /* 1/5! */
  p = p * r + 0x1.555556p-5f;   /* 1/4! */
  p = p * r + 0x1.555556p-3f;   /* 1/3! */
  p = p * r + 0.5f;
  p = p * r + 1.0f;
  p = p * r + 1.0f;
  const uint32_t tb = (uint32_t)((int)k + 127) << 23;
  float two_k;
  memcpy(&two_k, &tb, 4);
  return p * two_k;
}

/* cos(2 pi u) for u in [0, 1]: symmetries to w in [0, 1/4], then the Taylor series of
 * cos (angle <= pi/4, to a^10/10!) or of sin of the complement (to b^9/9!) */
float or_des_cos2pi(float u) {
  float v = u;
  if (v > 0.5f) v = 1.0f - v;
  float sign = 1.0f;
  if (v > 0.25f) {
    v = 0.5f - v;
    sign = -1.0f;
  }
  float c;
  if (v <= 0.125f) {
    const float a = 0x1.921fb6p+2f * v;
    const float a2 = a * a;
    float p = -0x1.27e4fcp-22f;   /* -1/10! */
    p = p * a2 + 0x1.a01a02p-16f; /* 1/8! */
    p = p * a2 - 0x1.6c16c2p-10f; /* 1/6! */
    p = p * a2 + 0x1.555556p-5f;  /* 1/4! */
    p = p * a2 - 0.5f;
    c = p * a2 + 1.0f;
  } else {
    const float bb = 0x1.921fb6p+2f * (0.25f - v);
    const float b2 = bb * bb;
    float p = 0x1.71de3ap-19f;    /* 1/9! */
    p = p * b2 - 0x1.a01a02p-13f; /* 1/7! */
    p = p * b2 + 0x1.111112p-7f;  /* 1/5! */
    p = p * b2 - 0x1.555556p-3f;  /* 1/3! */
    p = p * b2 + 1.0f;
    c = bb * p;
  }
  return sign * c;
}

/* one standard normal from two uniforms (Box-Muller, cosine branch) */
static float des_normal(float u1, float u2) {
  return sqrtf(-2.0f * or_des_ln(u1)) * or_des_cos2pi(u2);
}

/* a service time of mean m (FP32) */
float or_des_service(int kind, float m, uint64_t key, uint64_t c0) {
  const float u2 = des_u24(key, c0), u3 = des_u24(key, c0 + 1);
  switch (kind) {
    case 0:
      return -m * or_des_ln(u2);
    case 1: {
      const float s2 = 0x1.62e43p-1f; /* ln 2: the exponential's variance */
      const float mu = or_des_ln(m) - 0.5f * s2;
      return or_des_exp(mu + sqrtf(s2) * des_normal(u2, u3));
    }
    case 2: {
      float prod = u2 * u3;
      prod = prod * des_u24(key, c0 + 2);
      prod = prod * des_u24(key, c0 + 3);
      prod = prod * des_u24(key, c0 + 4);
      return -(m / 5.0f) * or_des_ln(prod);
    }
    case 3: {
      const float z = des_normal(u2, u3);
      return m * (z * z);
    }
    case 4:
      return (2.0f * m) * u2;
    default:
      return -1.0f;
  }
}

float or_des_uniform(uint64_t seed, int64_t r, uint64_t c) {
  return des_u24(des_mix(seed + (uint64_t)(r + 1) * DES_GAMMA), c);
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
  const float lamf = (float)lam;
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
      t = t + (double)(-or_des_ln(des_u24(key, c)) / lamf);
      const int in_window = a >= warmup;
      if (a == warmup) {
        /* the window opens: services in progress count from here */
        t0 = t;
        for (int i = 0; i < N; i++)
          if (fr[i] > t0) busy[r * N + i] = fr[i] - t0;
      }
      /* node: the first j whose cumulative rate reaches u lambda */
      const double target = des_u53(key, c + 1) * lam;
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
      const double s = (double)or_des_service(kind, (float)(1.0 / nu[unit]), key, c + 2);
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
