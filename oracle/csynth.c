/*
 * Test infrastructure only (part of the FP64 oracle): only tests/ may load
 * the library built from this file.  It shares no code with the CUDA path.
 *
 * The space integral of Eq. (1) in the frequency domain, written out plainly
 * for surveys whose reflection response is too large to hold as a dense FP64
 * array (the 4001-position survey: 984 x 4001 x 4001 complex values,
 * 252 GB):
 *
 *     S[m][k][f] = c * sum_r R_m(k, r) * N[m][r][f],
 *     R_m(k, r)  = T[m][|k - r|] * g[k][r],
 *
 * with R rebuilt element by element from the two factors the input
 * generator defines it by (T: offset spectra of the flat-layered primaries,
 * g: the reciprocal jitter scale).  Complex values are (re, im) pairs of
 * doubles.  The sum over r runs in increasing r, one accumulator per
 * (m, k, f); frequencies are shared out over threads, nothing else is
 * reordered or blocked.
 */
#include <pthread.h>
#include <stddef.h>
#include <stdint.h>

typedef struct {
  int nw, n, F, tid, nthreads;
  const double* T;  /* [nw][n] complex */
  const double* g;  /* [n][n] real */
  const double* N;  /* [nw][n][F] complex */
  double c;
  double* S;        /* [nw][n][F] complex */
} job_t;

enum { kMaxF = 64 };

static void* run(void* arg) {
  const job_t* j = (const job_t*)arg;
  const int n = j->n, F = j->F;
  for (int m = j->tid; m < j->nw; m += j->nthreads) {
    const double* Tm = j->T + (size_t)m * n * 2;
    const double* Nm = j->N + (size_t)m * n * F * 2;
    double* Sm = j->S + (size_t)m * n * F * 2;
    for (int k = 0; k < n; ++k) {
      const double* gk = j->g + (size_t)k * n;
      double acc[2 * kMaxF];
      for (int f = 0; f < 2 * F; ++f) acc[f] = 0.0;
      for (int r = 0; r < n; ++r) {
        const int o = k > r ? k - r : r - k;
        const double rr = Tm[2 * o] * gk[r], ri = Tm[2 * o + 1] * gk[r];  /* R_m(k, r) */
        const double* x = Nm + (size_t)r * F * 2;
        for (int f = 0; f < F; ++f) {
          acc[2 * f] += rr * x[2 * f] - ri * x[2 * f + 1];
          acc[2 * f + 1] += rr * x[2 * f + 1] + ri * x[2 * f];
        }
      }
      for (int f = 0; f < F; ++f) {
        Sm[((size_t)k * F + f) * 2] = j->c * acc[2 * f];
        Sm[((size_t)k * F + f) * 2 + 1] = j->c * acc[2 * f + 1];
      }
    }
  }
  return NULL;
}

/* Returns 0 on success, -1 for F outside 1 .. 64 or a thread that failed to start. */
int oracle_synthesis_factored(int nw, int n, int F, const double* T, const double* g, const double* N, double c,
                              double* S, int nthreads) {
  if (F < 1 || F > kMaxF || nw < 0 || n < 0) return -1;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  pthread_t th[256];
  job_t jobs[256];
  int started = 0, rc = 0;
  for (int t = 0; t < nthreads; ++t) {
    jobs[t] = (job_t){nw, n, F, t, nthreads, T, g, N, c, S};
    if (pthread_create(&th[t], NULL, run, &jobs[t]) != 0) {
      rc = -1;
      break;
    }
    ++started;
  }
  for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
  if (rc != 0) {  /* a thread did not start: finish its frequencies here */
    for (int t = started; t < nthreads; ++t) {
      jobs[t] = (job_t){nw, n, F, t, nthreads, T, g, N, c, S};
      run(&jobs[t]);
    }
  }
  return 0;
}
