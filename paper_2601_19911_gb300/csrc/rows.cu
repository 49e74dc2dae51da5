// Row-store helpers of the full-row offload, the foil of key-only transfer
// with late materialization (Sec. II-C; Sec. V-E measures both): whole rows
// cross the link, the key field is pulled out of every row on the device,
// and the selected rows are gathered there before they return.
#include "ctx.h"

namespace olap {

namespace {

// keys[i] = the W-byte field at rows + i * row_bytes + key_offset.  Aligned
// fields are read whole; otherwise byte by byte.
template <int W>
__global__ void rows_extract_kernel(const unsigned char* rows, uint64_t n, uint32_t row_bytes, uint32_t key_offset,
                                    unsigned char* keys, int aligned) {
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        const unsigned char* src = rows + i * row_bytes + key_offset;
        if (aligned) {
            if (W == 8) reinterpret_cast<uint64_t*>(keys)[i] = __ldcs(reinterpret_cast<const unsigned long long*>(src));
            else reinterpret_cast<uint32_t*>(keys)[i] = __ldcs(reinterpret_cast<const unsigned int*>(src));
        } else {
            for (int b = 0; b < W; ++b) keys[i * W + b] = src[b];
        }
    }
}

// out row j = rows row idx[j]; one warp per row, 4-byte words when rows and
// their length allow, else bytes.
__global__ void rows_gather_kernel(const unsigned char* rows, uint32_t row_bytes, const uint32_t* idx, uint64_t k,
                                   unsigned char* out, int words) {
    const uint64_t warps = static_cast<uint64_t>(gridDim.x) * (blockDim.x / 32);
    const unsigned lane = threadIdx.x & 31u;
    for (uint64_t j = static_cast<uint64_t>(blockIdx.x) * (blockDim.x / 32) + (threadIdx.x >> 5); j < k; j += warps) {
        const unsigned char* src = rows + static_cast<uint64_t>(idx[j]) * row_bytes;
        unsigned char* dst = out + j * row_bytes;
        if (words) {
            for (uint32_t b = lane; b < row_bytes / 4; b += 32)
                reinterpret_cast<uint32_t*>(dst)[b] = reinterpret_cast<const uint32_t*>(src)[b];
        } else {
            for (uint32_t b = lane; b < row_bytes; b += 32) dst[b] = src[b];
        }
    }
}

}  // namespace

cudaError_t rows_extract(const void* rows, uint64_t n, uint32_t row_bytes, uint32_t key_offset, int key_width,
                         void* keys, int grid, cudaStream_t s) {
    const uintptr_t base = reinterpret_cast<uintptr_t>(rows);
    const int aligned = ((base + key_offset) % key_width == 0 && row_bytes % key_width == 0) ? 1 : 0;
    const unsigned char* r = static_cast<const unsigned char*>(rows);
    unsigned char* kp = static_cast<unsigned char*>(keys);
    if (key_width == 8) rows_extract_kernel<8><<<grid, 256, 0, s>>>(r, n, row_bytes, key_offset, kp, aligned);
    else rows_extract_kernel<4><<<grid, 256, 0, s>>>(r, n, row_bytes, key_offset, kp, aligned);
    return cudaGetLastError();
}

cudaError_t rows_gather(const void* rows, uint32_t row_bytes, const uint32_t* idx, uint64_t k, void* out, int grid,
                        cudaStream_t s) {
    const int words = (reinterpret_cast<uintptr_t>(rows) % 4 == 0 && reinterpret_cast<uintptr_t>(out) % 4 == 0 &&
                       row_bytes % 4 == 0)
                          ? 1
                          : 0;
    rows_gather_kernel<<<grid, 256, 0, s>>>(static_cast<const unsigned char*>(rows), row_bytes, idx, k,
                                            static_cast<unsigned char*>(out), words);
    return cudaGetLastError();
}

}  // namespace olap
