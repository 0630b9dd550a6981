// Reads cases "kind args... expected" from stdin and compares the library's
// SU(2) coefficients (su2.cpp) with them; every case is evaluated twice so
// that the second value comes from the coefficient memo.  Prints the largest
// absolute error per kind; exits 1 if any exceeds 1e-12.
#include <cmath>
#include <cstdio>
#include <map>
#include <string>

#include "su2.hpp"

int main() {
  char kind[16];
  std::map<std::string, double> worst;
  int n = 0;
  while (std::scanf("%15s", kind) == 1) {
    int v[9] = {0};
    double want = 0.0, got1 = 0.0, got2 = 0.0;
    const std::string k = kind;
    const int na = k == "6j" ? 6 : k == "cg" ? 6 : 9;
    for (int i = 0; i < na; ++i)
      if (std::scanf("%d", &v[i]) != 1) return 2;
    if (std::scanf("%lf", &want) != 1) return 2;
    for (int rep = 0; rep < 2; ++rep) {
      double g = 0.0;
      if (k == "6j") g = dmrg::wigner6j(v[0], v[1], v[2], v[3], v[4], v[5]);
      else if (k == "9j") g = dmrg::wigner9j(v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7], v[8]);
      else if (k == "cg") g = dmrg::clebsch(v[0], v[1], v[2], v[3], v[4], v[5]);
      else if (k == "tp") g = dmrg::tensor_product_coef(v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7], v[8]);
      else return 2;
      (rep ? got2 : got1) = g;
    }
    if (got1 != got2) {
      std::printf("memo changed the value of %s case %d\n", kind, n);
      return 1;
    }
    worst[k] = std::fmax(worst[k], std::fabs(got1 - want));
    ++n;
  }
  bool ok = n > 0;
  for (auto& [k, e] : worst) {
    std::printf("%s max abs error %.3e\n", k.c_str(), e);
    ok = ok && e <= 1e-12;
  }
  std::printf("%d cases\n", n);
  return ok ? 0 : 1;
}
