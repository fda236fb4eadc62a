// Applies dd.cuh's double-double operations to operands read from stdin, one
// per line: "<op> a_hi a_lo b_hi b_lo" with op in add, mul, mul_d (b = b_hi),
// recip (a only), two_prod (a_hi * b_hi); prints "hi lo" (17 significant digits).
#include <cstdio>
#include <cstring>

#include "dd.cuh"

int main() {
  char op[16];
  double ah, al, bh, bl;
  while (std::scanf("%15s %lf %lf %lf %lf", op, &ah, &al, &bh, &bl) == 5) {
    const rplu::dd a{ah, al}, b{bh, bl};
    rplu::dd r{0.0, 0.0};
    if (!std::strcmp(op, "add")) r = rplu::dd_add(a, b);
    else if (!std::strcmp(op, "mul")) r = rplu::dd_mul(a, b);
    else if (!std::strcmp(op, "mul_d")) r = rplu::dd_mul_d(a, bh);
    else if (!std::strcmp(op, "recip")) r = rplu::dd_recip(a);
    else if (!std::strcmp(op, "two_prod")) r = rplu::two_prod(ah, bh);
    else return 2;
    std::printf("%.17g %.17g\n", r.hi, r.lo);
  }
  return 0;
}
