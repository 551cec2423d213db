/* Using the C ABI of include/vmc.h directly: a batch of walkers on the n = 216
 * simple-cubic system (kappa 2, r_c 1.5), two Metropolis sweeps with logs, one
 * single move with its drift quantities, the kinetic energy of every walker, and the
 * solver statistics.  Build against the in-tree library, e.g.
 *   gcc vmc_sweep_example.c -I../../include -L.. -lvmc -Wl,-rpath,$PWD/.. -o example
 * Exit status 0 when every call succeeds and the logs are consistent. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "vmc.h"

#define WALKERS 4
#define CHECK(call)                                                                \
  do {                                                                             \
    vmc_status s_ = (call);                                                        \
    if (s_ != VMC_OK) {                                                            \
      fprintf(stderr, "%s failed (%d): %s\n", #call, (int)s_, vmc_last_error(ctx)); \
      return 1;                                                                    \
    }                                                                              \
  } while (0)

int main(void) {
  vmc_system sys[WALKERS];
  uint64_t seeds[WALKERS];
  for (int w = 0; w < WALKERS; ++w) {
    sys[w].K = 6;
    sys[w].lattice = 0;
    sys[w].a = 1.0;
    sys[w].kappa = 2.0;
    sys[w].r_c = 1.5;
    seeds[w] = (uint64_t)(w + 1);
  }
  vmc_solver_params p;
  vmc_ctx* ctx = NULL;
  CHECK(vmc_default_params(&p));
  CHECK(vmc_create(sys, WALKERS, &p, NULL, &ctx));
  CHECK(vmc_init_positions(ctx, seeds, 0.1));

  const int n = vmc_walker_n(ctx, 0), sweeps = 2;
  const size_t entries = (size_t)sweeps * n * WALKERS;
  uint8_t* acc = (uint8_t*)malloc(entries);
  double* ratio = (double*)malloc(entries * sizeof(double));
  CHECK(vmc_sweep(ctx, sweeps, 0.2, seeds, acc, ratio));
  size_t accepted = 0;
  for (size_t e = 0; e < entries; ++e) {
    if (!isfinite(ratio[e])) return 2;
    accepted += acc[e];
  }

  /* a single move of walker 0's particle 5, with the drift quantities at r' */
  double R[3 * 216];
  CHECK(vmc_get_positions(ctx, 0, R));
  const double r_new[3] = {R[15] + 0.1, R[16] - 0.05, R[17] + 0.02};
  double rat = 0.0, grad[3], lap = 0.0;
  CHECK(vmc_ratio_grad(ctx, 0, 5, r_new, &rat, grad, &lap));
  CHECK(vmc_accept(ctx, 0));

  double energy[WALKERS];
  CHECK(vmc_kinetic_energy(ctx, energy));

  vmc_stats st;
  CHECK(vmc_get_stats(ctx, 0, &st));
  printf("n=%d walkers=%d sweeps=%d accepted=%zu ratio=%.6f grad=(%.4f %.4f %.4f) lap=%.4f "
         "E_kin[0]=%.6f solves=%lld factorizations=%lld async_lag=%d\n",
         n, WALKERS, sweeps, accepted, rat, grad[0], grad[1], grad[2], lap, energy[0], (long long)st.solves,
         (long long)st.factorizations, st.async_lag);
  CHECK(vmc_destroy(ctx));
  free(acc);
  free(ratio);
  return (accepted > 0 && st.proposals == (int64_t)sweeps * n + 1) ? 0 : 3;
}
