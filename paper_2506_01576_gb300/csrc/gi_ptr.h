// How the C ABI treats a caller's pointer, as a pure function of what the CUDA
// runtime reports for it (host-only, no CUDA headers, so it is tested on the CPU).
//
//   device memory of the index's own device ...... used in place
//   managed memory ............................... used in place (any device can reach it)
//   host memory (registered, or unknown to CUDA) . staged through device buffers
//   device memory of ANOTHER device .............. refused: a kernel launched on the
//                                                  index's device would read a
//                                                  foreign address (without peer
//                                                  access, an illegal-address fault)
#pragma once

namespace gi {

enum PtrClass { kPtrDevice = 0, kPtrHost = 1, kPtrRefused = 2 };

// type: the cudaMemoryType of the pointer's attributes (0 unregistered, 1 host,
//       2 device, 3 managed), or -1 when the attribute query failed (memory the
//       runtime does not know: pageable host memory);
// ptr_device: the attributes' device; want_device: the index's device.
inline PtrClass classify_pointer(int type, int ptr_device, int want_device) {
  switch (type) {
    case 2:
      return ptr_device == want_device ? kPtrDevice : kPtrRefused;
    case 3:
      return kPtrDevice;
    default:
      return kPtrHost;
  }
}

}  // namespace gi
