// Host driver for the CPU checks of the double-word header (csrc/dword.cuh): reads one
// operation per line from stdin, operands as hexadecimal IEEE 754 bit patterns, and
// prints the result bits.  Built with g++ -ffp-contract=off by tests/test_dword.py.
//   W f            -> widen_f(f)                     (binary32 -> binary64)
//   S x            -> dw_of(x).hi dw_of(x).lo        (binary64 -> double word)
//   T hi lo        -> dw_to_double({hi, lo})
//   A ah al bh bl  -> dw_add(a, b)
//   M ah al bh bl  -> dw_mul(a, b)
//   F ah al b      -> dw_mulf(a, b)
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "paper_2602_17950_gb300/csrc/dword.cuh"

using gpsoc::DF;

static float F(unsigned long long u) { return gpsoc::f_from((unsigned)u); }
static DF D(unsigned long long h, unsigned long long l) {
  DF r;
  r.hi = F(h);
  r.lo = F(l);
  return r;
}
static unsigned long long dbits(double x) {
  unsigned long long b;
  memcpy(&b, &x, 8);
  return b;
}

int main() {
  char op[4];
  while (scanf("%3s", op) == 1) {
    unsigned long long a = 0, b = 0, c = 0, d = 0;
    if (op[0] == 'W') {
      if (scanf("%llx", &a) != 1) return 2;
      printf("%016llx\n", dbits(gpsoc::widen_f(F(a))));
    } else if (op[0] == 'S') {
      if (scanf("%llx", &a) != 1) return 2;
      double x;
      memcpy(&x, &a, 8);
      const DF r = gpsoc::dw_of(x);
      printf("%08x %08x\n", gpsoc::f_bits(r.hi), gpsoc::f_bits(r.lo));
    } else if (op[0] == 'T') {
      if (scanf("%llx %llx", &a, &b) != 2) return 2;
      printf("%016llx\n", dbits(gpsoc::dw_to_double(D(a, b))));
    } else if (op[0] == 'F') {
      if (scanf("%llx %llx %llx", &a, &b, &c) != 3) return 2;
      const DF r = gpsoc::dw_mulf(D(a, b), F(c));
      printf("%08x %08x\n", gpsoc::f_bits(r.hi), gpsoc::f_bits(r.lo));
    } else {
      if (scanf("%llx %llx %llx %llx", &a, &b, &c, &d) != 4) return 2;
      const DF r = (op[0] == 'A') ? gpsoc::dw_add(D(a, b), D(c, d)) : gpsoc::dw_mul(D(a, b), D(c, d));
      printf("%08x %08x\n", gpsoc::f_bits(r.hi), gpsoc::f_bits(r.lo));
    }
  }
  return 0;
}
