/* A plain C client of include/hmc.h: links libhmc.so and calls the entry
 * points that need no GPU (sizes, filter and rooted-polynomial coefficients,
 * argument checks), printing the results one per line for the test that
 * compares them with the oracle's exact series.  Builds as C99. */
#include <stdio.h>

#include "hmc.h"

int main(void) {
  hmc_lattice lat = {{48, 24, 24, 24}};
  printf("spinor_bytes_f32 %zu\n", hmc_spinor_bytes(&lat, HMC_F32, 1));
  printf("gauge_bytes_f32_12 %zu\n", hmc_gauge_bytes(&lat, HMC_F32, HMC_LINK12));
  printf("algebra_bytes %zu\n", hmc_algebra_bytes(&lat));
  hmc_lattice odd = {{48, 24, 24, 23}};
  printf("spinor_bytes_odd %zu\n", hmc_spinor_bytes(&odd, HMC_F64, 1));

  double b[30], c[30], alpha = 0.0;
  int st = hmc_filter_coeffs(2, 29, b, &alpha, c);
  printf("filter_status %d\n", st);
  printf("filter_alpha %.17g\n", alpha);
  for (int n = 0; n <= 29; ++n) printf("filter_b %d %.17g\n", n, b[n]);
  for (int n = 0; n <= 29; ++n) printf("filter_c %d %.17g\n", n, c[n]);
  printf("filter_bad %d\n", hmc_filter_coeffs(9, 29, b, &alpha, c));

  const int degrees[2] = {6, 12};
  double rb[21], polys[7 + 13], ralpha = 0.0;
  st = hmc_rooted_coeffs(2, 2, 2, degrees, 20, &ralpha, rb, polys);
  printf("rooted_status %d\n", st);
  printf("rooted_alpha %.17g\n", ralpha);
  for (int i = 0; i < 20; ++i) printf("rooted_poly %d %.17g\n", i, polys[i]);

  printf("null_ctx %d\n", hmc_ctx_set_option(NULL, HMC_OPT_PDL, 1));
  printf("null_ctx_error %s\n", hmc_last_error(NULL));
  return 0;
}
