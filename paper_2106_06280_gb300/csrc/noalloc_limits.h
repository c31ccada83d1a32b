// Size limit of the allocation-free conservation sums (cswdg_conservation_noalloc):
// the reduction's per-block partial sums live in one fixed device array of
// NOALLOC_MAX_BLOCKS x NOALLOC_MAX_VARS doubles (2 MiB), 256 cells per block.
// Plain host C++ with no CUDA dependency, so the check can be compiled and
// exercised on its own.
#ifndef CSW_NOALLOC_LIMITS_H
#define CSW_NOALLOC_LIMITS_H
#include <stdint.h>

#define CSW_NOALLOC_CELLS_PER_BLOCK 256
#define CSW_NOALLOC_MAX_BLOCKS 65536  // at most 16,777,216 cells
#define CSW_NOALLOC_MAX_VARS 4

// true when nc cells of nvar variables fit the fixed scratch
static inline bool csw_noalloc_fits(int64_t nc, int nvar)
{
    if (nc < 1 || nvar < 1 || nvar > CSW_NOALLOC_MAX_VARS) return false;
    const int64_t nblk = (nc + CSW_NOALLOC_CELLS_PER_BLOCK - 1) / CSW_NOALLOC_CELLS_PER_BLOCK;
    return nblk <= CSW_NOALLOC_MAX_BLOCKS;
}
#endif
