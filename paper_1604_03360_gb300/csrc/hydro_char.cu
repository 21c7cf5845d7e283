// hydro_char.cu -- instantiations of the characteristic-wise stage kernels
// (global Lax-Friedrichs split, WENO on the characteristic fields): the fused
// stage kernel and the face passes (char_pass.cuh) + stage_combine_kernel.
#include "char_pass.cuh"
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

// x, y and z face passes (one thread per face, MINB CTAs per SM) and the
// per-cell combination
template <int R, int NF, int EMU, int MINB>
static cudaError_t char_pass_info(StageLaunch* out)
{
    void (*fns[3])(StageArgs) = {charw_pass_kernel<R, NF, 0, EMU, MINB>, charw_pass_kernel<R, NF, 1, EMU, MINB>,
                                 charw_pass_kernel<R, NF, 2, EMU, MINB>};
    const size_t smem = char_pass_smem<R, NF>();
    for (int d = 0; d < 3; ++d) {
        const cudaError_t e = cudaFuncSetAttribute(fns[d], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    out->xfn = fns[0];
    out->yfn = fns[1];
    out->zfn = fns[2];
    out->fn = stage_combine_kernel<NF, false>;
    out->combine = true;
    out->face_per_thread = true;
    out->pass_threads = kCharPassThreads;
    out->pass_smem = smem;
    out->smem = 0;
    out->tx = 16;
    out->ty = 16;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&out->ctas_per_sm, stage_combine_kernel<NF, false>, 256, 0);
}

// Fused stage kernel: WENO5 0 16x16 (196 KB shared memory) and 1 16x8;
// WENO7 0 16x8 (16x16 would need 247 KB); several charges 0 16x8.
// Face passes (then the combination), numbered after those: products with
// constants on the integer pipe, at three and at four CTAs per SM (12 and 16
// warps), and at four CTAs per SM with the weight products there too.
// 256^3 ellipsoidal stage: WENO7 123.9 / 125.3 / 133.5 ms (fused 16x8: 161.7),
// WENO5 81.5 / 82.4 / 78.1 ms (fused 16x8: 104.0).
int char_variant_count(int R, int nq)
{
    return (nq > 1 || R == 4 ? 1 : 2) + 3;
}

// the default: the face passes, WENO5 with the weight products on the integer
// pipe (256^3: 78.1 against 81.5 ms), WENO7 without (123.9 against 133.5 ms)
int char_default_variant(int R, int nq)
{
    return (nq > 1 || R == 4 ? 1 : 2) + (R == 3 ? 2 : 0);
}

template <int R, int NF>
static cudaError_t char_pass_variant(int v, StageLaunch* out)
{
    if (v == 0) return char_pass_info<R, NF, kEmuConst, 3>(out);
    if (v == 1) return char_pass_info<R, NF, kEmuConst, 4>(out);
    if (v == 2) return char_pass_info<R, NF, kEmuConst | kEmuWeights, 4>(out);
    return cudaErrorInvalidValue;
}

cudaError_t char_launch_variant(int R, int nq, int v, StageLaunch* out)
{
    if (R != 3 && R != 4) return cudaErrorInvalidValue;
    const int nfused = nq > 1 || R == 4 ? 1 : 2;
    if (v >= nfused) {
        if (nq == 2) return R == 3 ? char_pass_variant<3, 6>(v - nfused, out) : char_pass_variant<4, 6>(v - nfused, out);
        if (nq == 3) return R == 3 ? char_pass_variant<3, 7>(v - nfused, out) : char_pass_variant<4, 7>(v - nfused, out);
        return R == 3 ? char_pass_variant<3, 5>(v - nfused, out) : char_pass_variant<4, 5>(v - nfused, out);
    }
    if (nq > 1) {
        if (nq == 2) return R == 3 ? char_info_for<3, 16, 8, 6>(out) : char_info_for<4, 16, 8, 6>(out);
        if (nq == 3) return R == 3 ? char_info_for<3, 16, 8, 7>(out) : char_info_for<4, 16, 8, 7>(out);
        return cudaErrorInvalidValue;
    }
    if (R == 3) {
        if (v == 0) return char_info_for<3, 16, 16, 5>(out);
        return char_info_for<3, 16, 8, 5>(out);
    }
    return char_info_for<4, 16, 8, 5>(out);
}

}  // namespace hydro
