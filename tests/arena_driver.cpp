// Drives the server's first-fit arena bookkeeping (offsets only) from stdin for the CPU tests:
//   c <capacity>   reset        -> prints capacity
//   a <bytes>      allocate     -> prints offset or -1
//   f <offset>     release      -> prints 1 / 0
// after every command also prints: used largest_free free_blocks live_blocks
#include <stdio.h>

#include "../paper_1706_02740_gb300/csrc/arena.h"

int main() {
  sft::OffsetArena A;
  char op;
  long long v;
  while (scanf(" %c %lld", &op, &v) == 2) {
    long long r = 0;
    if (op == 'c') {
      A.reset((size_t)v);
      r = (long long)A.capacity();
    } else if (op == 'a') {
      r = (long long)A.alloc((size_t)v);
    } else if (op == 'f') {
      r = A.release((size_t)v) ? 1 : 0;
    }
    printf("%lld %zu %zu %zu %zu\n", r, A.used(), A.largest_free(), A.free_blocks(), A.live_blocks());
  }
  return 0;
}
