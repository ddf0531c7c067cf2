// Tensor maps of the dense-box stage path (see cmx_dense.cuh), built on the host for each launch
// from the buffers of the launch's context: 4-D tensors (x, y, z, component) over the dense
// (nz, ny, nxs) arrays, out-of-box positions filled with zero.
#include <cuda.h>

#include "cmx_dense.cuh"
#include "cmx_kernels.h"

namespace cmx {

namespace {

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                 const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                 const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's cuTensorMapEncodeTiled, looked up once through the runtime (no link against
// libcuda).
EncodeTiled encoder()
{
    static EncodeTiled fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

// Map of `base` seen as (nx, ny, nz, ncomp) FP32 with rows of nxs cells, planes of nxs ny cells
// and components ncell apart, read in boxes of bx x by x 1 x ncomp.
cudaError_t encode(EncodeTiled enc, CUtensorMap *m, const void *base, const Ctx &c, int ncomp,
                   int bx, int by, CUtensorMapL2promotion promo)
{
    const cuuint64_t dim[4] = {(cuuint64_t)c.nx, (cuuint64_t)c.ny, (cuuint64_t)c.nz,
                               (cuuint64_t)ncomp};
    const cuuint64_t stride[3] = {(cuuint64_t)c.nxs * 4, (cuuint64_t)c.nxs * c.ny * 4,
                                  (cuuint64_t)c.ncell * 4};
    const cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, 1u, (cuuint32_t)ncomp};
    const cuuint32_t es[4] = {1u, 1u, 1u, 1u};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void *>(base), dim,
                           stride, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, promo,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

cudaError_t build_dense_maps(const Ctx &c, int wy, void *map, int count)
{
    if (count < TM_COUNT || !map) return cudaErrorInvalidValue;
    // the dense layout: rows of nxs >= nx cells (a multiple of 8, so every stride is a multiple
    // of 16 bytes), exactly nz ny rows per component
    if (c.nxs < c.nx || c.nxs % 8 != 0 || (long long)c.ncell != (long long)c.nxs * c.ny * c.nz)
        return cudaErrorInvalidValue;
    EncodeTiled enc = encoder();
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap *m = static_cast<CUtensorMap *>(map);
    const int nq = 3 * c.nsub;
    const int tx = DX, ty = wy + 2, ox = 32, oy = wy;
    cudaError_t e = cudaSuccess;
    // L2 fills: the tile boxes' rows (160 bytes from a 16-byte offset) in 128-byte lines; the
    // operand rows (128 bytes, aligned) without promotion, since the neighbouring tile's half of
    // a wider line is read by another block much later and mostly evicted by then
    auto put = [&](int i, const void *base, int ncomp, int bx, int by) {
        const CUtensorMapL2promotion promo = bx == DX ? CU_TENSOR_MAP_L2_PROMOTION_L2_128B
                                                      : CU_TENSOR_MAP_L2_PROMOTION_NONE;
        if (e == cudaSuccess && base) e = encode(enc, &m[i], base, c, ncomp, bx, by, promo);
    };
    for (int b = 0; b < 2; b++) {
        put(TMT_M + b, c.m[b], nq, tx, ty);
        put(TMT_MSV + b, c.msv[b], nq, tx, ty);
        put(TMO_M + b, c.m[b], nq, ox, oy);
    }
    for (int j = 0; j < 7; j++) {
        put(TMT_K + j, c.k[j], nq, tx, ty);
        put(TMO_K + j, c.k[j], nq, ox, oy);
    }
    put(TMO_ES, c.es, nq, ox, oy);
    if (c.u && c.nmodes > 0) put(TMO_U, c.u, c.nmodes, ox, oy);
    return e;
}

}  // namespace cmx
