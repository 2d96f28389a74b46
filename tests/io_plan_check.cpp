// The chunk plan of the host-buffer calls (flame_init_f32_host,
// flame_moments_f32_host), checked for every plane count up to 600, for
// periodic lattices and z-slabs: the copy chunks and the initialisation
// chunks partition their planes with none empty; each initialisation chunk
// waits for a copy chunk at or after every chunk holding one of the planes
// its central differences read (a - 1 .. b, periodic); and the last
// initialisation waits for the last copy.  Prints the counts, exits non-zero
// on a violation.
#include <cstdio>
#include <cstdlib>
#include "flame_internal.h"
using namespace flame;
int main() {
  long bad = 0, cases = 0;
  for (int nz = 1; nz <= 600; ++nz)
    for (int slab = 0; slab < 2; ++slab) {
      if (slab && nz < 3) continue;
      const int z0 = slab ? 1 : 0, nzi = slab ? nz - 2 : nz;
      const int nc = io_chunk_count(nz), ni = io_chunk_count(nzi);
      if (nc < 1 || nc > kIoChunks || ni < 1 || ni > kIoChunks) { ++bad; continue; }
      // copy chunks partition [0, nz), none empty
      if (io_first(0, nz, nc, 0) != 0 || io_first(0, nz, nc, nc) != nz) ++bad;
      for (int j = 0; j < nc; ++j) if (io_first(0, nz, nc, j + 1) <= io_first(0, nz, nc, j)) ++bad;
      for (int q = 0; q < nz; ++q) {
        int j = io_chunk_of(nz, nc, q);
        if (!(io_first(0, nz, nc, j) <= q && q < io_first(0, nz, nc, j + 1))) ++bad;
      }
      // init chunks partition [z0, z0 + nzi)
      if (io_first(z0, nzi, ni, 0) != z0 || io_first(z0, nzi, ni, ni) != z0 + nzi) ++bad;
      int maxneed = -1;
      for (int j = 0; j < ni; ++j) {
        const int a = io_first(z0, nzi, ni, j), b = io_first(z0, nzi, ni, j + 1);
        if (b <= a || a < 0 || b > nz) ++bad;
        const int need = io_init_needs(nz, nc, a, b);
        if (need < 0 || need >= nc) ++bad;
        if (need > maxneed) maxneed = need;
        for (int p = a - 1; p <= b; ++p) {
          const int q = ((p % nz) + nz) % nz;
          if (io_chunk_of(nz, nc, q) > need) ++bad;
        }
        ++cases;
      }
      if (maxneed != nc - 1) { ++bad; printf("maxneed nz=%d slab=%d %d %d\n", nz, slab, maxneed, nc); }
    }
  printf("cases %ld bad %ld\n", cases, bad);
  return bad != 0;
}
