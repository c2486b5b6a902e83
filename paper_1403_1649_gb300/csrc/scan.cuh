// scan.cuh -- device-wide exclusive prefix sum (three passes: tile scan,
// scan of tile totals, add).  Deterministic; used for CSR row pointers, root
// numbering and aggregate member offsets.
#pragma once
#include "amg_internal.cuh"

namespace amg {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// out[i] = sum_{k<i} in[k] inside each tile of kScanTile items; tile totals to sums
template <class TI, class TO>
__global__ void k_scan_tiles(const TI *__restrict__ in, TO *__restrict__ out, int64_t n,
                             TO *__restrict__ sums) {
  pdl_wait_and_trigger();
  __shared__ TO warp_tot[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  TO v[kScanItems];
  TO run = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + k;
    TO x = (i < n) ? (TO)in[i] : (TO)0;
    v[k] = run;
    run += x;
  }
  // exclusive scan of per-thread totals across the block
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  TO incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    TO y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    TO t = (lane < kScanThreads / 32) ? warp_tot[lane] : (TO)0;
    TO ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      TO y = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += y;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = ti - t;  // exclusive
    if (lane == kScanThreads / 32 - 1) sums[blockIdx.x] = ti;
  }
  __syncthreads();
  const TO off = warp_tot[wid] + (incl - run);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + k;
    if (i < n) out[i] = v[k] + off;
  }
}

template <class TO>
__global__ void k_scan_add(TO *__restrict__ out, int64_t n, const TO *__restrict__ sums) {
  pdl_wait_and_trigger();
  const TO add = sums[blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  for (int k = threadIdx.x; k < kScanTile; k += blockDim.x) {
    int64_t i = base + k;
    if (i < n) out[i] += add;
  }
}

// Exclusive scan of n items; out has n+1 entries, out[n] = total.  Returns the
// total (synchronises the stream to read it back when want_total is set).
template <class TI, class TO>
void exclusive_scan(const TI *in, TO *out, int64_t n, cudaStream_t s, TO *total_host = nullptr) {
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (n == 0) {
    AMG_CUDA(cudaMemsetAsync(out, 0, sizeof(TO), s));
    if (total_host) *total_host = 0;
    return;
  }
  DevBuf<TO> sums(tiles + 1);
  AMG_COUNT(), klaunch_sm(k_scan_tiles<TI, TO>, (unsigned)tiles, kScanThreads, 0, s, in, out, n, sums.p);
  AMG_LAUNCH_CHECK();
  if (tiles > 1) {
    DevBuf<TO> ssc(tiles + 1);
    exclusive_scan<TO, TO>(sums.p, ssc.p, tiles, s, nullptr);
    AMG_COUNT(), klaunch_sm(k_scan_add<TO>, (unsigned)tiles, kScanThreads, 0, s, out, n, ssc.p);
    AMG_LAUNCH_CHECK();
    // out[n] = last exclusive value + last input = total
    AMG_CUDA(cudaMemcpyAsync(out + n, ssc.p + tiles, sizeof(TO), cudaMemcpyDeviceToDevice, s));
  } else {
    AMG_CUDA(cudaMemcpyAsync(out + n, sums.p, sizeof(TO), cudaMemcpyDeviceToDevice, s));
  }
  if (total_host) {
    AMG_CUDA(cudaMemcpyAsync(total_host, out + n, sizeof(TO), cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaStreamSynchronize(s));
  }
}

}  // namespace amg
