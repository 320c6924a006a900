// match_tc.h -- the tensor-core matching kernel (match_tc.cu) as seen by
// match.cu: BF16 centred images, K padded to a multiple of 64, the k best
// model images per scene image.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/spin.h"

namespace si {

constexpr int kMatchTcMaxK = 16;       // k best per scene image, at most
constexpr int kMatchTcMaxParts = 32;   // model ranges per scene block, at most

// Model ranges per scene block that fill whole waves of `sms` SMs best.
int match_tc_parts(int64_t n_scene, int64_t n_model, int sms);

// a: [n_scene][kp], b: [n_model][kp] (BF16, rows 16-byte aligned, kp % 64 == 0);
// part_v / part_i: [2 parts][n_scene][k] scratch; err: a zeroed device word.
// Writes best_idx / best_val [n_scene][k]; if a bounded device wait gave up,
// every best_idx of the call is -2.
si_status match_tc_launch(const __nv_bfloat16 *a, int64_t n_scene, const __nv_bfloat16 *b, int64_t n_model, int kp,
                          int k, int parts, float *part_v, int *part_i, unsigned *err, int32_t *best_idx,
                          float *best_val, cudaStream_t st);

}  // namespace si
