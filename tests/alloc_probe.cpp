// Host-only: prints the key-array sizes of csrc/gi_alloc.h for the (n, key bytes,
// eytzinger) triples read from stdin, one "used alloc" line each.
#include <cstdio>

#include "gi_alloc.h"

int main() {
  unsigned long long n;
  int kb, eytz;
  while (std::scanf("%llu %d %d", &n, &kb, &eytz) == 3)
    std::printf("%llu %llu\n", (unsigned long long)gi::key_used_bytes(n, kb, eytz != 0),
                (unsigned long long)gi::key_alloc_bytes(n, kb));
  return 0;
}
