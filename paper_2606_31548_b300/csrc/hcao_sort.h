// hcao_sort.h -- stable counting sort by cell key (device buffers).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hcao {
constexpr int SORT_TILE = 256 * 8;  // keys per CTA tile
// scratch words (uint32) cell_sort needs for n keys
int64_t sort_scratch_words(int64_t n, uint32_t n_cells);
int sort_passes(uint32_t n_cells);
// keys[n] < n_cells -> perm[n] (input index of each sorted position, equal keys
// in input order), offsets[n_cells + 1] (start of each cell).  All device.
cudaError_t cell_sort(const uint32_t* keys, int64_t n, uint32_t n_cells, uint32_t* perm,
                      uint32_t* offsets, uint32_t* scratch, cudaStream_t s, uint64_t* launches);
}  // namespace hcao
