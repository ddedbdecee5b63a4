// Per-device record of kernel attributes already applied (host-only C++,
// no CUDA dependency, so it is unit-tested on the CPU).
//
// A kernel's dynamic-shared-memory limit (cudaFuncAttributeMaxDynamicSharedMemorySize)
// is a property of the kernel on one device: setting it while device 0 is
// current leaves the kernel at the 48 KB default on device 1.  The library
// therefore remembers, per (kernel, device ordinal), the largest limit it has
// set, and sets it again whenever a launch on a device needs more.  Lookups
// and updates hold a mutex, so host threads driving different devices (or
// the same one) may launch concurrently.
#pragma once

#include <stddef.h>

#include <map>
#include <mutex>
#include <utility>

namespace ibmk {

class DeviceAttrTable {
  public:
    // Run `apply` (which sets the attribute and returns 0 on success) unless
    // a limit of at least `bytes` is already recorded for (func, device).
    // Records `bytes` only when `apply` succeeds; returns apply's code or 0.
    template <typename Apply>
    int ensure(const void *func, int device, size_t bytes, Apply apply) {
        std::lock_guard<std::mutex> lock(mu_);
        const auto key = std::make_pair(func, device);
        auto it = done_.find(key);
        if (it != done_.end() && it->second >= bytes) return 0;
        const int rc = apply();
        if (rc != 0) return rc;
        done_[key] = bytes;
        return 0;
    }

    // the recorded limit, 0 if none (for tests)
    size_t recorded(const void *func, int device) {
        std::lock_guard<std::mutex> lock(mu_);
        auto it = done_.find(std::make_pair(func, device));
        return it == done_.end() ? 0 : it->second;
    }

  private:
    std::mutex mu_;
    std::map<std::pair<const void *, int>, size_t> done_;
};

}  // namespace ibmk
