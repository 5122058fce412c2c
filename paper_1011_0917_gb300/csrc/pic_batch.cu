// pic_batch.cu -- the particle kernels of a batch of runs: a persistent
// grid whose CTAs take (run, tile) items of all runs from a device-wide
// counter, each tile processed by the single-run kernels' body
// (pic_push.cuh) with its run's arguments.
#include "pic_push.cuh"

namespace pic {

// The particle kernels of a batch of runs: a persistent grid whose CTAs take
// (run, tile) work items from a device-wide counter until all are done, each
// tile processed as by push_kernel / ion_kernel with its run's arguments
// (copied into shared memory when the run changes).
template <typename real, int DIM, int S, int TX, int TY, int TZ, bool REL, bool IONS>
__device__ __forceinline__ void batch_tiles(const PushArgs<real> *__restrict__ runs, const int64_t *__restrict__ start,
                                            int n, unsigned *queue, unsigned char *smem_raw)
{
    __shared__ __align__(16) PushArgs<real> sa;
    __shared__ int64_t s_item;
    __shared__ int s_run;
    const int64_t total = start[n];
    int cur = -1;
    // thread 0 claims the next item while the CTA works on the current one,
    // and looks the run up only when the item leaves the last run's range
    int64_t next = 0, run_lo = 0, run_hi = 0;
    int run = -1;
    if (threadIdx.x == 0) next = (int64_t)atomicAdd(queue, 1u);
    for (;;) {
        if (threadIdx.x == 0) {
            const int64_t item = next;
            if (item < total) {
                if (item < run_lo || item >= run_hi) {
                    run = batch_run_of(start, n, item);
                    run_lo = start[run];
                    run_hi = start[run + 1];
                }
                next = (int64_t)atomicAdd(queue, 1u);
            }
            s_item = item;
            s_run = item < total ? run : -1;
        }
        __syncthreads();
        const int r = s_run;
        if (r < 0) break;
        const int64_t t = s_item - start[r];
        if (r != cur) {
            batch_copy_args(&sa, runs + r);
            cur = r;
            __syncthreads();
        }
        if (IONS) ion_tile<real, DIM, S, TX, TY, TZ, REL>(sa, t, smem_raw);
        else push_tile<real, DIM, S, TX, TY, TZ, REL>(sa, t, smem_raw);
        __syncthreads();  // (an empty tile returns at once) every thread has read s_item, s_run
    }
}

template <typename real, int DIM, int S, int TX, int TY, int TZ, bool REL>
__global__ void __launch_bounds__(kBlock, MinBlocks<real>::value)
    push_batch_kernel(const PushArgs<real> *__restrict__ runs, const int64_t *__restrict__ start, int n,
                      unsigned *queue)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    batch_tiles<real, DIM, S, TX, TY, TZ, REL, false>(runs, start, n, queue, smem_raw);
}

template <typename real, int DIM, int S, int TX, int TY, int TZ, bool REL>
__global__ void __launch_bounds__(kBlock)
    ion_batch_kernel(const PushArgs<real> *__restrict__ runs, const int64_t *__restrict__ start, int n,
                     unsigned *queue)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    batch_tiles<real, DIM, S, TX, TY, TZ, REL, true>(runs, start, n, queue, smem_raw);
}

// batched form: a persistent grid of as many CTAs as fit on the device
template <typename real, int DIM, int S, int TX, int TY, int TZ, bool REL, bool IONS>
void launch_push_batch(const void *args, const int64_t *start, int n, int64_t total, unsigned *queue,
                              cudaStream_t s)
{
    const size_t smem = push_smem<real, DIM, S, TX, TY, TZ, REL>(IONS);
    auto k = IONS ? ion_batch_kernel<real, DIM, S, TX, TY, TZ, REL> : push_batch_kernel<real, DIM, S, TX, TY, TZ, REL>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kBlock, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    int64_t grid = (int64_t)per_sm * device_sms();
    if (grid > total) grid = total;
    if (grid < 1) grid = 1;
    k<<<(unsigned)grid, kBlock, smem, s>>>(static_cast<const PushArgs<real> *>(args), start, n, queue);
}

// every kernel configuration the single-run launchers dispatch to
template void launch_push_batch<float, 3, 1, 8, 8, 8, true, true>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<float, 3, 1, 8, 8, 8, true, false>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<float, 3, 1, 8, 8, 8, false, true>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<float, 3, 1, 8, 8, 8, false, false>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<float, 3, 2, 8, 8, 8, true, true>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<float, 3, 2, 8, 8, 8, true, false>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<float, 3, 2, 8, 8, 8, false, true>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<float, 3, 2, 8, 8, 8, false, false>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<float, 2, 2, 16, 1, 16, true, true>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<float, 2, 2, 16, 1, 16, true, false>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<float, 2, 2, 16, 1, 16, false, true>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<float, 2, 2, 16, 1, 16, false, false>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<float, 2, 1, 32, 1, 8, true, true>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<float, 2, 1, 32, 1, 8, true, false>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<float, 2, 1, 32, 1, 8, false, true>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<float, 2, 1, 32, 1, 8, false, false>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<float, 2, 1, 8, 1, 32, true, true>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<float, 2, 1, 8, 1, 32, true, false>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<float, 2, 1, 8, 1, 32, false, true>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<float, 2, 1, 8, 1, 32, false, false>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<float, 2, 1, 16, 1, 16, true, true>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<float, 2, 1, 16, 1, 16, true, false>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<float, 2, 1, 16, 1, 16, false, true>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<float, 2, 1, 16, 1, 16, false, false>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<double, 3, 1, 8, 8, 8, true, true>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<double, 3, 1, 8, 8, 8, true, false>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<double, 3, 1, 8, 8, 8, false, true>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<double, 3, 1, 8, 8, 8, false, false>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<double, 3, 2, 8, 8, 8, true, true>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<double, 3, 2, 8, 8, 8, true, false>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<double, 3, 2, 8, 8, 8, false, true>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<double, 3, 2, 8, 8, 8, false, false>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<double, 2, 2, 16, 1, 16, true, true>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<double, 2, 2, 16, 1, 16, true, false>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<double, 2, 2, 16, 1, 16, false, true>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<double, 2, 2, 16, 1, 16, false, false>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<double, 2, 1, 32, 1, 8, true, true>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<double, 2, 1, 32, 1, 8, true, false>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<double, 2, 1, 32, 1, 8, false, true>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<double, 2, 1, 32, 1, 8, false, false>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<double, 2, 1, 8, 1, 32, true, true>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<double, 2, 1, 8, 1, 32, true, false>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<double, 2, 1, 8, 1, 32, false, true>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<double, 2, 1, 8, 1, 32, false, false>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<double, 2, 1, 16, 1, 16, true, true>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<double, 2, 1, 16, 1, 16, true, false>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<double, 2, 1, 16, 1, 16, false, true>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<double, 2, 1, 16, 1, 16, false, false>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);

template void launch_push_batch<float, 3, 1, 8, 8, 4, true, true>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<float, 3, 1, 8, 8, 4, true, false>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<float, 3, 1, 8, 8, 4, false, true>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<float, 3, 1, 8, 8, 4, false, false>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<double, 3, 1, 8, 8, 4, true, true>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<double, 3, 1, 8, 8, 4, true, false>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<double, 3, 1, 8, 8, 4, false, true>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);
template void launch_push_batch<double, 3, 1, 8, 8, 4, false, false>(const void *, const int64_t *, int, int64_t, unsigned *, cudaStream_t);

}  // namespace pic
