/*
 * ne_probe.h -- throughput probes of the benchmark (libne_probe.so), kept out
 * of the library's ABI (include/ne.h): each launches a register-resident loop
 * of one instruction kind on every SM of the current device, on stream s, and
 * writes the number of operations it issues to *ops (host pointer).  The
 * caller times the launch with events on s; operations / time is the
 * instruction's ceiling, the denominator of a kernel's roofline fraction.
 * Returns NE_PROBE_OK, NE_PROBE_EINVAL (arguments) or NE_PROBE_ECUDA (launch).
 */
#ifndef NE_PROBE_H
#define NE_PROBE_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NE_PROBE_OK 0
#define NE_PROBE_EINVAL 1
#define NE_PROBE_ECUDA 3

/* mma.sync.m16n8k32 s8 (the int8 tensor instruction of sm_103a): int8
 * operations (2 per multiply-add).  iters >= 1. */
int32_t ne_probe_mma_peak(int32_t iters, int64_t* ops, cudaStream_t s);

/* dp4a on the CUDA cores (four int8 products added into an int32): int8
 * operations.  iters >= 1. */
int32_t ne_probe_dp4a_peak(int32_t iters, int64_t* ops, cudaStream_t s);

/* 32-bit integer multiply-add (IMAD): multiply-adds.  iters >= 1. */
int32_t ne_probe_imad_peak(int32_t iters, int64_t* ops, cudaStream_t s);

/* Both int8 pipes in one launch: blocks_per_sm blocks per SM (1..8), each
 * with mma_warps warps of the tensor loop (iters_mma rounds) and dp4a_warps
 * warps of the dp4a loop (iters_dp4a rounds), 1..16 warps in all: the
 * ceiling of a kernel that splits its work between the pipes in that ratio.
 * *ops: the int8 operations of both. */
int32_t ne_probe_mixed_peak(int32_t iters_mma, int32_t iters_dp4a, int32_t mma_warps, int32_t dp4a_warps,
                            int32_t blocks_per_sm, int64_t* ops, cudaStream_t s);

#ifdef __cplusplus
}
#endif

#endif /* NE_PROBE_H */
