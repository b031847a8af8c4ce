// Host-only check of gi::classify_pointer (csrc/gi_ptr.h): how the C ABI treats
// a pointer given what the CUDA runtime reports for it.  Prints one line per case.
#include <cstdio>

#include "gi_ptr.h"

int main() {
  struct Case {
    int type, ptr_dev, want_dev, expect;
    const char* what;
  } cases[] = {
      {2, 0, 0, gi::kPtrDevice, "device memory of the index's device"},
      {2, 3, 3, gi::kPtrDevice, "device memory of the index's device (device 3)"},
      {2, 1, 0, gi::kPtrRefused, "device memory of another device"},
      {2, 0, 1, gi::kPtrRefused, "device memory of another device (reversed)"},
      {3, 1, 0, gi::kPtrDevice, "managed memory"},
      {1, 0, 0, gi::kPtrHost, "registered host memory"},
      {1, 2, 0, gi::kPtrHost, "registered host memory reported with another device"},
      {0, -1, 0, gi::kPtrHost, "unregistered host memory"},
      {-1, -1, 0, gi::kPtrHost, "memory unknown to the runtime"},
  };
  int bad = 0;
  for (const Case& c : cases) {
    const int got = gi::classify_pointer(c.type, c.ptr_dev, c.want_dev);
    std::printf("%s: %s\n", c.what, got == c.expect ? "ok" : "WRONG");
    bad += got != c.expect;
  }
  return bad ? 1 : 0;
}
