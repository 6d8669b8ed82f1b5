// rtlfs_static.h -- the allocation-free fault-simulation variant (rtlfs_static.cu).
#pragma once
#include "rtlfs_internal.h"

namespace rtlfs {

// Size of the file-scope device scratch array used by rtlfs_fault_sim_static.
constexpr size_t STATIC_SCRATCH_BYTES = (size_t)64 << 20;
constexpr int STATIC_MAX_DEVICES = 64;

// Same layouts as rtlfs_fault / rtlfs_result of include/rtlfs.h.
struct StaticFault {
    uint32_t net;
    uint8_t bit, stuck;
    uint16_t reserved;
};
struct StaticResult {
    int32_t cycle, port;
    uint8_t detected, reserved[3];
};

// Offsets (bytes) into the scratch array and per-thread strides (elements).
struct StaticLayout {
    size_t ext2int_off, err_off, thread_off, per_thread;
    uint32_t sn, snode, sreg;
};

// Device address of the scratch array on `device` (looked up once per device).
cudaError_t static_scratch_address(int device, void **out);
cudaError_t launch_plain_static(const DevDesign *d_designs, uint32_t design, const void *faults,
                                void *results, uint32_t first, uint32_t count, void *arena,
                                StaticLayout L, cudaStream_t stream);

}  // namespace rtlfs
