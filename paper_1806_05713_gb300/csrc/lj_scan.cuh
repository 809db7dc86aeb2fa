// lj_scan.cuh -- exclusive prefix sums used by the pair-list builder (the
// counting sort that groups atoms by cell and list entries by row).
#pragma once

#include "lj_internal.cuh"

namespace lj {

constexpr int kScanBlock = 512;
constexpr int kScanItems = 8;
constexpr int64_t kScanChunk = int64_t(kScanBlock) * kScanItems;

// Per-chunk exclusive scan: out[k] = sum of in[chunk start .. k-1];
// chunk_sums[b] = sum of the chunk (64-bit).  Summation in 64 bits.
template <class Tin, class Tout>
__global__ void __launch_bounds__(kScanBlock)
scan_chunks_kernel(const Tin *__restrict__ in, Tout *__restrict__ out, int64_t n,
                   int64_t *__restrict__ chunk_sums)
{
    __shared__ long long warp_tot[kScanBlock / 32];
    const int64_t base = int64_t(blockIdx.x) * kScanChunk + int64_t(threadIdx.x) * kScanItems;
    long long v[kScanItems];
    long long s = 0;
#pragma unroll
    for (int t = 0; t < kScanItems; ++t) {
        const int64_t k = base + t;
        v[t] = k < n ? static_cast<long long>(in[k]) : 0;
        s += v[t];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        long long w = lane < kScanBlock / 32 ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kScanBlock / 32) warp_tot[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    long long run = incl - s + (warp > 0 ? warp_tot[warp - 1] : 0);
#pragma unroll
    for (int t = 0; t < kScanItems; ++t) {
        const int64_t k = base + t;
        if (k < n) out[k] = static_cast<Tout>(run);
        run += v[t];
    }
    if (threadIdx.x == kScanBlock - 1) chunk_sums[blockIdx.x] = run;
}

template <class Tout>
__global__ void scan_add_kernel(Tout *__restrict__ out, int64_t n,
                                const int64_t *__restrict__ chunk_offsets)
{
    const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k < n) out[k] = static_cast<Tout>(static_cast<long long>(out[k]) + chunk_offsets[k / kScanChunk]);
}

__global__ void scan_total_kernel(const int64_t *__restrict__ chunk_offsets,
                                  const int64_t *__restrict__ chunk_sums, int64_t nchunks,
                                  int64_t *__restrict__ total)
{
    *total = nchunks > 0 ? chunk_offsets[nchunks - 1] + chunk_sums[nchunks - 1] : 0;
}

// Scratch (int64 words) that scan_exclusive needs for n items.
inline size_t scan_scratch_words(int64_t n)
{
    size_t words = 0;
    int64_t m = n;
    while (true) {
        const int64_t chunks = (m + kScanChunk - 1) / kScanChunk;
        words += 2 * size_t(chunks > 0 ? chunks : 1) + 5;
        if (chunks <= 1) break;
        m = chunks;
    }
    return words + 8;
}

// out[k] = in[0] + ... + in[k-1] for k < n; *total_dev = sum of all n.
// Summation is exact in 64 bits; Tout may truncate (callers check the total).
template <class Tin, class Tout>
int scan_exclusive(const Tin *in, Tout *out, int64_t n, int64_t *total_dev, int64_t *scratch,
                   cudaStream_t st)
{
    if (n <= 0) {
        LJ_TRY_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(int64_t), st));
        return LJ_OK;
    }
    const int64_t chunks = (n + kScanChunk - 1) / kScanChunk;
    int64_t *sums = scratch;
    int64_t *offs = scratch + chunks;
    int64_t *rest = offs + chunks + 4;
    scan_chunks_kernel<Tin, Tout><<<unsigned(chunks), kScanBlock, 0, st>>>(in, out, n, sums);
    LJ_TRY_LAUNCH("scan_chunks_kernel");
    if (chunks == 1) {
        LJ_TRY_CUDA(cudaMemcpyAsync(total_dev, sums, sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
        return LJ_OK;
    }
    int rc = scan_exclusive<int64_t, int64_t>(sums, offs, chunks, rest, rest + 1, st);
    if (rc != LJ_OK) return rc;
    scan_add_kernel<Tout><<<unsigned((n + 255) / 256), 256, 0, st>>>(out, n, offs);
    LJ_TRY_LAUNCH("scan_add_kernel");
    scan_total_kernel<<<1, 1, 0, st>>>(offs, sums, chunks, total_dev);
    LJ_TRY_LAUNCH("scan_total_kernel");
    return LJ_OK;
}

}  // namespace lj
