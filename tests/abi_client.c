/* A plain C99 client of libstark.so, built and run by tests/test_abi.py on a
 * machine without a GPU: the header must compile as C (not only C++) and the
 * host-only entry points must link and answer.  It prints, on one line: the
 * status and C-target counts of the depth-1 quadrant table (Alg. 1's
 * C11..C22 over M1..M7), then the server admission of an n = 1024 FP64
 * request under an ample budget (status, depth, levels, bytes), then the
 * text of STARK_ENOMEM. */
#include <stdio.h>

#include "stark.h"

int main(void) {
  int32_t count[7], quad[7 * 2];
  int8_t sign[7 * 2];
  int32_t depth = -1, levels = -1;
  int64_t bytes = 0;
  int i;
  stark_status t = stark_quadrant_table(1, 2, count, quad, sign);
  stark_status a = stark_server_admission((size_t)1 << 40, 1024, STARK_F64, 0, &depth, &levels, &bytes);
  printf("%d", (int)t);
  for (i = 0; i < 7; ++i) printf(" %d", (int)count[i]);
  printf(" %d %d %d %lld %s\n", (int)a, (int)depth, (int)levels, (long long)bytes, stark_strerror(STARK_ENOMEM));
  return 0;
}
