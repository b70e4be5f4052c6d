// The GPU engine of the level loop's Schur complements (schur_gpu.cu).
#pragma once
#include <cuda_runtime.h>

#include <memory>

#include "ildl_setup.h"

namespace ajd {

// A SchurEngine on the current device whose work runs on stream `st`.
std::unique_ptr<SchurEngine> make_device_schur(cudaStream_t st);

}  // namespace ajd
