// sw_align_batch_noalloc: the scan-F batch alignment without any device
// allocation, for callers that cannot let a library allocate device memory
// (for example an application whose own allocator has reserved the device's
// memory, or a host framework that forbids its plug-ins to allocate).
//
// All scratch of the call -- the length-binned work order, the zeroed
// counters, the overflow list of packed lanes and the chunk boundary rows of
// long queries -- lives in one file-scope device array of
// SW_NOALLOC_SCRATCH_BYTES, which every GPU that loads the library keeps
// until the process exits.  Every call reuses that one array, so calls whose
// work overlaps on the GPU (on different streams, or issued from different
// host threads) race and must be serialised by the caller.  The counters
// that have to start at zero are cleared by each call on its stream.
//
// The first call on a device looks up the array's device address with
// cudaGetSymbolAddress (with that device current); make that first call
// before any stream capture.  Host code must never pass the array's name to
// a kernel: on the host it only stands for the device object.
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "sw_gb300.h"
#include "sw_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[SW_NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;
void *g_scratch_ptr[64] = {nullptr};

// device address of the scratch array on the current device (looked up once)
int scratch_address(int dev, void **out)
{
    if (dev < 0 || dev >= 64)
        return swg::api_fail(SW_ERR_INVALID, "sw_align_batch_noalloc: device index out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (err != cudaSuccess)
            return swg::api_cuda_fail((int)err, "cudaGetSymbolAddress(no-allocation scratch)");
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return SW_OK;
}

size_t align_256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

extern "C" int sw_align_batch_noalloc(const sw_profile *prof, const uint8_t *db, const int64_t *off, int64_t n_db,
                                      int32_t o, int32_t e, int32_t *scores, void *cuda_stream)
{
    int rc = swg::api_check_align_args(prof, db, off, n_db, o, e, scores);
    if (rc)
        return rc;
    if (n_db == 0)
        return SW_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (prof->qlen == 0) {
        const cudaError_t err = cudaMemsetAsync(scores, 0, sizeof(int32_t) * (size_t)n_db, st);
        return err == cudaSuccess ? SW_OK : swg::api_cuda_fail((int)err, "cudaMemsetAsync");
    }
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != prof->device)
        return swg::api_fail(SW_ERR_INVALID, "profile built on another device than the current one");
    void *base = nullptr;
    rc = scratch_address(dev, &base);
    if (rc)
        return rc;
    const int sms = swg::api_num_sms(dev);

    int lane = prof->lane;
    if (lane != SW_LANE_I32 && !swg::api_lane_fits(lane, prof, o, e, prof->plan))
        lane = SW_LANE_I32;
    const swg::Plan main = lane == SW_LANE_I32 ? prof->plan32 : prof->plan;
    const int8_t *main_prof = lane == SW_LANE_I32 ? prof->d_prof32 : prof->d_prof;
    const bool packed = lane != SW_LANE_I32;
    const int C32 = prof->plan32.C;
    const bool chunked = main.C > 1 || (packed && C32 > 1);
    int64_t total = 0;
    if (chunked) {  // boundary rows are sized by the residue count
        cudaError_t err = cudaMemcpyAsync(&total, off + n_db, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
        if (err == cudaSuccess)
            err = cudaStreamSynchronize(st);
        if (err != cudaSuccess)
            return swg::api_cuda_fail((int)err, "reading db_offsets[n_db]");
        if (total < 0)
            return swg::api_fail(SW_ERR_INVALID, "db_offsets[n_db] < 0");
    }
    const size_t n = (size_t)n_db;
    const int ncount = main.C + (packed ? C32 : 0) + 2;
    const size_t sz_order = align_256(n * 4);
    const size_t sz_zero = align_256((2 * swg::NBINS + ncount) * 4);
    const size_t sz_list = packed ? align_256(n * 4) : 0;
    const size_t sz_bnd = chunked ? align_256((size_t)total * sizeof(int2) + 16) : 0;
    const size_t need = sz_order + sz_zero + sz_list + sz_bnd;
    if (need > (size_t)SW_NOALLOC_SCRATCH_BYTES) {
        char msg[256];
        snprintf(msg, sizeof(msg),
                 "sw_align_batch_noalloc: this call needs %zu bytes of scratch, the fixed array holds %zu "
                 "(%lld sequences, %lld residues)",
                 need, (size_t)SW_NOALLOC_SCRATCH_BYTES, (long long)n_db, (long long)total);
        return swg::api_fail(SW_ERR_RANGE, msg);
    }
    char *p = (char *)base;
    int32_t *order = (int32_t *)p;
    int32_t *zero = (int32_t *)(p + sz_order);
    int32_t *bins = zero;
    uint32_t *counters = (uint32_t *)(zero + 2 * swg::NBINS);
    int32_t *list_count = (int32_t *)(counters + main.C + (packed ? C32 : 0));
    int32_t *list = (int32_t *)(p + sz_order + sz_zero);
    int2 *bnd = chunked ? (int2 *)(p + sz_order + sz_zero + sz_list) : nullptr;

    // the array keeps the previous call's contents: clear what counts from 0
    cudaError_t err = cudaMemsetAsync(zero, 0, sz_zero, st);
    if (err != cudaSuccess)
        return swg::api_cuda_fail((int)err, "cudaMemsetAsync(no-allocation scratch)");
    int kr = swg::launch_length_order(off, n_db, order, bins, st, sms);
    if (kr)
        return swg::api_cuda_fail(kr, "length order kernels");

    swg::BatchArgs a;
    memset(&a, 0, sizeof(a));
    a.A = prof->A;
    a.qlen = prof->qlen;
    a.db = db;
    a.off = off;
    a.order = order;
    a.n_work = n_db;
    a.o = o;
    a.e = e;
    a.bnd = bnd;
    a.scores = scores;
    a.one = 1;
    a.flag_thresh = swg::api_flag_threshold(lane, o, prof->maxM);
    a.min_m = prof->minM;
    a.prof = main_prof;
    a.nchunks = main.C;
    for (int c = 0; c < main.C; ++c) {
        a.chunk = c;
        a.counter = counters + c;
        kr = swg::api_launch_plan(main, false, a, sms, st);
        if (kr)
            return swg::api_cuda_fail(kr, "batch kernel launch");
    }
    if (packed) {
        kr = swg::launch_flag_overflow(scores, n_db, a.flag_thresh, list, list_count, st, sms);
        if (kr)
            return swg::api_cuda_fail(kr, "overflow flag kernel");
        a.prof = prof->d_prof32;
        a.flag_thresh = INT32_MAX;
        a.nchunks = C32;
        a.order = list;
        a.n_work = n_db;
        a.n_work_dev = list_count;
        for (int c = 0; c < C32; ++c) {
            a.chunk = c;
            a.counter = counters + main.C + c;
            kr = swg::api_launch_plan(prof->plan32, false, a, sms, st);
            if (kr)
                return swg::api_cuda_fail(kr, "rescore kernel launch");
        }
    }
    return SW_OK;
}
