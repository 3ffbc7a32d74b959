// fe_persist_wait_selftest: the bounded wait of the persistent trial
// launch's tile claim, run where no tile ever becomes available and no trial
// is ever decided, so that a test can check that the wait gives up (and
// raises the launch's abort flag) instead of spinning on.
#include <cuda_runtime.h>

#include "fe_internal.cuh"
#include "fe_tile_common.cuh"

namespace fe {
namespace {

// One warp claims a tile from one image whose only tile is already taken
// (sched = ntiles), with one image still counted active and no decision to
// come: persist_grab waits out its limit and returns -1.
__global__ void persist_wait_selftest_kernel(KParams p, int *result) {
    int pref = 0;
    const int t = persist_grab(p, pref);
    if (threadIdx.x == 0) *result = t;
}

}  // namespace
}  // namespace fe

using namespace fe;

extern "C" fe_status fe_persist_wait_selftest(double stall_s, int *aborted, double *waited_s) {
    if (!aborted || !waited_s || !(stall_s > 0.0) || stall_s > 5.0) return FE_EINVAL;
    *aborted = -1;
    *waited_s = 0.0;
    struct Buf {
        ImgDesc img;
        LoopCtl lc;
        int sched, porder, result, pad;
    };
    Buf h{};
    h.img.H = h.img.W = 64;
    h.img.tile_begin = 0;
    h.img.ntiles = 1;
    h.lc.active = 1;
    h.sched = 1;  // the image's one tile is taken: nothing to claim
    h.porder = 0;
    h.result = -2;
    Buf *d = nullptr;
    if (cudaMalloc(&d, sizeof(Buf)) != cudaSuccess) return FE_ENOMEM;
    fe_status st = FE_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.f;
    KParams p{};
    p.imgs = &d->img;
    p.loop = &d->lc;
    p.sched = &d->sched;
    p.porder = &d->porder;
    p.nimg = 1;
    p.persist_stall_ns = (unsigned long long)(stall_s * 1e9);
    if (cudaMemcpy(d, &h, sizeof(Buf), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        st = FE_ECUDA;
    } else {
        cudaEventRecord(e0);
        persist_wait_selftest_kernel<<<1, 32>>>(p, &d->result);
        cudaEventRecord(e1);
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
            cudaMemcpy(&h, d, sizeof(Buf), cudaMemcpyDeviceToHost) != cudaSuccess)
            st = FE_ECUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(d);
    if (st != FE_OK) return st;
    *aborted = (h.result == -1 && h.lc.abort == 1) ? 1 : 0;
    *waited_s = 1e-3 * ms;
    return *aborted ? FE_ETIMEOUT : FE_OK;
}
