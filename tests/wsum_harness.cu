// Host harness for the predictor's integer weighted sum (wsum_int in
// lb_device.cuh, compiled here from the same source through lb_grid.cu).
// Reads lines "n x_0 ... x_{n-1}" with every x_i as the hexadecimal bit
// pattern of a double (x_0 the oldest ring entry) and prints the bit pattern
// of the weighted sum, one per line.  n is 8, 9 or 10.
#include "../paper_2110_10310_gb300/csrc/lb_grid.cu"

#include <cinttypes>
#include <cstdio>

int main() {
  int n = 0;
  while (std::scanf("%d", &n) == 1) {
    double x[10];
    for (int i = 0; i < n && i < 10; ++i) {
      unsigned long long u = 0;
      if (std::scanf("%llx", &u) != 1) return 2;
      std::memcpy(&x[i], &u, sizeof u);
    }
    double r = 0.0;
    switch (n) {
      case 8: r = lbk::wsum_int<8>(*reinterpret_cast<double(*)[8]>(x)); break;
      case 9: r = lbk::wsum_int<9>(*reinterpret_cast<double(*)[9]>(x)); break;
      case 10: r = lbk::wsum_int<10>(x); break;
      default: return 3;
    }
    unsigned long long b = 0;
    std::memcpy(&b, &r, sizeof b);
    std::printf("%016llx\n", b);
  }
  return 0;
}
