// Host driver for the region-wise plane-fit inverse of the CUDA path
// (fsl::plic_alpha_regions): reads "tv m1 m2 m3" lines, prints the float and
// double results.  Built and run by tests/test_plic_regions.py.
#include <cstdio>

#include "fslbm_dev.cuh"

int main() {
  double tv, m1, m2, m3;
  while (std::scanf("%lf %lf %lf %lf", &tv, &m1, &m2, &m3) == 4) {
    const float af = fsl::plic_alpha_regions<float>((float)tv, (float)m1, (float)m2, (float)m3);
    const double ad = fsl::plic_alpha_regions<double>(tv, m1, m2, m3);
    std::printf("%.9g %.17g\n", (double)af, ad);
  }
  return 0;
}
