// hydro_char.cu -- instantiations of the characteristic-wise stage kernel
// (global Lax-Friedrichs split, WENO on the characteristic fields).
#include "hydro_common.cuh"

namespace hydro {

template <int R, int TX, int TY, int NF>
static cudaError_t char_info_for(StageLaunch* out)
{
    auto fn = stage_kernel<R, TX, TY, 1, false, NF, true>;
    out->fn = fn;
    out->zfn = nullptr;
    out->smem = StageSmem<R, TX, TY, false, NF, true>::bytes;
    out->tx = TX;
    out->ty = TY;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)out->smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&out->ctas_per_sm, fn, TX * TY, out->smem);
}

// WENO5: 16x16 (196 KB shared memory) and 16x8; WENO7: 16x8 (16x16 would
// need 247 KB); several charges: 16x8.
int char_variant_count(int R, int nq)
{
    if (nq > 1) return 1;
    return R == 3 ? 2 : 1;
}

cudaError_t char_launch_variant(int R, int nq, int v, StageLaunch* out)
{
    if (R != 3 && R != 4) return cudaErrorInvalidValue;
    if (nq > 1) {
        if (v != 0) return cudaErrorInvalidValue;
        if (nq == 2) return R == 3 ? char_info_for<3, 16, 8, 6>(out) : char_info_for<4, 16, 8, 6>(out);
        if (nq == 3) return R == 3 ? char_info_for<3, 16, 8, 7>(out) : char_info_for<4, 16, 8, 7>(out);
        return cudaErrorInvalidValue;
    }
    if (R == 3) {
        if (v == 0) return char_info_for<3, 16, 16, 5>(out);
        if (v == 1) return char_info_for<3, 16, 8, 5>(out);
        return cudaErrorInvalidValue;
    }
    if (v == 0) return char_info_for<4, 16, 8, 5>(out);
    return cudaErrorInvalidValue;
}

}  // namespace hydro
