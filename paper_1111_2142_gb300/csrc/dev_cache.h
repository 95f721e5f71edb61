// Per-device caches of one-time kernel set-up results (occupancy-derived grid
// sizes, shared-memory opt-ins). Kernel attributes and SM counts belong to a
// device, so a process that drives several GPUs keeps one value per device;
// the slots are atomic, so concurrent first calls from several host threads at
// worst compute the same value twice.
#pragma once

#include <cuda_runtime.h>

#include <atomic>

namespace lwacm {

constexpr int kMaxDevices = 64;
using DevSlots = std::atomic<int>[kMaxDevices];

// fn() -> int (0 is reserved for "not yet known"), cached for the current device
template <typename F>
inline int per_device(DevSlots &slots, F fn) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return fn();
    int v = slots[dev].load(std::memory_order_acquire);
    if (v == 0) {
        v = fn();
        slots[dev].store(v, std::memory_order_release);
    }
    return v;
}

// SM count of the current device (152 if it cannot be read)
inline int device_sms() {
    static DevSlots slots;
    return per_device(slots, [] {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0)
            return n;
        return 152;
    });
}

}  // namespace lwacm
