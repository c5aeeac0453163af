// dvm_readback.cuh -- pipelined read-back of the moments of a handle or a
// batch (dvm_moments_async / dvm_moments_wait and the batch pair): the
// moments and the status word are snapshotted on the device in stream order
// into one of two slots, and copied from there into the caller's buffer on a
// private copy stream while later steps run.
#pragma once

#include <cuda_runtime.h>

namespace dvm {

struct ReadBack {
  static constexpr int kRing = 64;  // tickets whose status is kept apart
  cudaStream_t copy = nullptr;
  double* snap = nullptr;           // 2 slots of `stride` doubles
  long long stride = 0;             // n moments + 2 (status word at the end)
  cudaEvent_t snap_ev[2] = {nullptr, nullptr};
  int* status = nullptr;            // pinned, status of ticket t at [t % kRing]
  cudaEvent_t ev[kRing] = {};       // ticket t's copies done
  long long issued = 0;

  // First use: the two slots (2 (n + 2) doubles), the ring, the copy stream.
  cudaError_t init(long long n) {
    cudaError_t e;
    stride = n + 2;
    if ((e = cudaMalloc(&snap, sizeof(double) * 2 * stride)) != cudaSuccess) return e;
    if ((e = cudaMallocHost(&status, kRing * sizeof(int))) != cudaSuccess) return e;
    for (int i = 0; i < kRing; ++i) status[i] = 0;
    if ((e = cudaStreamCreateWithFlags(&copy, cudaStreamNonBlocking)) != cudaSuccess) return e;
    for (int i = 0; i < 2; ++i)
      if ((e = cudaEventCreateWithFlags(&snap_ev[i], cudaEventDisableTiming)) != cudaSuccess) return e;
    for (int i = 0; i < kRing; ++i)
      if ((e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming)) != cudaSuccess) return e;
    return cudaSuccess;
  }

  // Read-back of the n moments at U and the status word at dstatus, after the
  // work enqueued on s so far, into out.
  cudaError_t issue(cudaStream_t s, const double* U, long long n, const int* dstatus, double* out,
                    bool on_device, long long* ticket) {
    cudaError_t e;
    if (!snap && (e = init(n)) != cudaSuccess) return e;
    const long long t = issued;
    const int slot = (int)(t & 1), r = (int)(t % kRing);
    double* sl = snap + slot * stride;
    // the slot's previous user, ticket t - 2, has been copied out of it
    if (t >= 2 && (e = cudaStreamWaitEvent(s, ev[(t - 2) % kRing], 0)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(sl, U, sizeof(double) * n, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(sl + n, dstatus, sizeof(int), cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(snap_ev[slot], s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(copy, snap_ev[slot], 0)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(out, sl, sizeof(double) * n,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, copy)) != cudaSuccess)
      return e;
    if ((e = cudaMemcpyAsync(status + r, sl + n, sizeof(int), cudaMemcpyDeviceToHost, copy)) != cudaSuccess)
      return e;
    if ((e = cudaEventRecord(ev[r], copy)) != cudaSuccess) return e;
    *ticket = t;
    issued = t + 1;
    return cudaSuccess;
  }

  // Waits for ticket (0 <= ticket < issued) and gives the status its snapshot
  // found.  A ticket whose ring entry a later one took waits for the newest
  // read-back instead (copies complete in ticket order, the status is sticky).
  cudaError_t wait(long long ticket, int* st) {
    const long long t = ticket < issued - kRing ? issued - 1 : ticket;
    const cudaError_t e = cudaEventSynchronize(ev[t % kRing]);
    if (e == cudaSuccess) *st = status[t % kRing];
    return e;
  }

  void release() {
    if (copy) {
      cudaStreamSynchronize(copy);
      cudaStreamDestroy(copy);
    }
    for (int i = 0; i < 2; ++i)
      if (snap_ev[i]) cudaEventDestroy(snap_ev[i]);
    for (int i = 0; i < kRing; ++i)
      if (ev[i]) cudaEventDestroy(ev[i]);
    if (snap) cudaFree(snap);
    if (status) cudaFreeHost(status);
  }
};

}  // namespace dvm
