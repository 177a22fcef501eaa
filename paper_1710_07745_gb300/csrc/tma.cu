// tma.cu -- host-side TMA tensor-map encoding for uint8 images.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "canny_internal.cuh"

namespace canny {

namespace {
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_once;

void resolve()
{
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    else
        cudaGetLastError();
}
}  // namespace

bool tma_usable(const void *base, int pitch)
{
    return (((uintptr_t)base) & 15) == 0 && (pitch & 15) == 0;
}

// 2-D map over an h x w uint8 image with the given pitch, box box_w x box_h;
// reads outside the image return 0.
bool encode_u8_map(void *tmap_out, const void *base, int w, int h, int pitch, int box_w, int box_h)
{
    std::call_once(g_once, resolve);
    if (!g_encode || !tma_usable(base, pitch)) return false;
    cuuint64_t dims[2] = {(cuuint64_t)w, (cuuint64_t)h};
    cuuint64_t strides[1] = {(cuuint64_t)pitch};
    cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode((CUtensorMap *)tmap_out, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(base),
                          dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace canny
