// Internal interfaces between the translation units of libmvsk.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "rowpass.cuh"

namespace mvsk {

enum Prec : int { P64 = 0, P16 = 1, P32 = 2 };

// Shared-memory bytes and ring stages for a pass; returns 0 when the shape
// (precision, mode, inputs, ld) is unsupported or does not fit.
size_t rowpass_smem(int prec, int mode, int nin, int ld, int* stages);

// Launch one streaming pass (grid CTAs, kThreads threads each).
cudaError_t rowpass_launch(int prec, int mode, int nin, const PassArgs& args, int grid, size_t smem,
                           cudaStream_t st);

// Per-precision dispatchers (one translation unit each).
size_t rowpass_smem_f64(int mode, int nin, int ld, int* stages);
size_t rowpass_smem_f32(int mode, int nin, int ld, int* stages);
size_t rowpass_smem_bf16(int mode, int nin, int ld, int* stages);
cudaError_t rowpass_init_f64();
cudaError_t rowpass_init_f32();
cudaError_t rowpass_init_bf16();
cudaError_t rowpass_launch_f64(int mode, int nin, const PassArgs& a, int grid, size_t smem, cudaStream_t st);
cudaError_t rowpass_launch_f32(int mode, int nin, const PassArgs& a, int grid, size_t smem, cudaStream_t st);
cudaError_t rowpass_launch_bf16(int mode, int nin, const PassArgs& a, int grid, size_t smem, cudaStream_t st);

// Text returned by mvsk_last_error (thread-local).
void set_last_error(const char* msg);

constexpr size_t kSmemBudget = 225 * 1024;  // dynamic; static shared memory needs the rest of 227 KB

}  // namespace mvsk
