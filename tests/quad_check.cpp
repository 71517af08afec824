// Prints the Gauss-Jacobi rules the device kernels get from the host
// (gauss_jacobi_rule): for each "n alpha beta" line on stdin, n lines of
// "node weight" with full precision.
#include <cstdio>
#include <vector>

#include "hfsem_internal.h"

int main() {
  int n;
  double al, be;
  while (std::scanf("%d %lf %lf", &n, &al, &be) == 3) {
    std::vector<double> x, w;
    hf::gauss_jacobi_rule(n, al, be, x, w);
    for (int i = 0; i < n; ++i) std::printf("%.17g %.17g\n", x[i], w[i]);
  }
  return 0;
}
