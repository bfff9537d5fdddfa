// Host-side check of the CommUp tiling (cu_box, cu_chunks in internal.h) against a
// brute-force enumeration: for every shape, ghost width and field, the tiles cover
// exactly the coarse hosts with a fine ghost among their 8 children, once each; every
// tile fits the kernel's shared-memory buffers; every halo stays in the range of
// hosts whose coarse stencil lies inside the parent; and the launch's chunk count is
// the number of tiles.  Prints "OK <tiles>" and exits 0, or "FAIL ..." and exits 1.
#include <cstdio>
#include <set>
#include <tuple>

#include "internal.h"

using namespace dfn;

int main() {
  const int shapes[][3] = {{8, 8, 8},    {24, 24, 24}, {64, 64, 64},   {128, 128, 128},
                           {12, 12, 24}, {32, 32, 64}, {48, 24, 96},   {200, 16, 16},
                           {16, 200, 16}, {16, 16, 200}, {36, 20, 44}};
  const int ghosts[] = {2, 4, 8, 16};
  long long tiles = 0;
  int bad = 0;
  for (const auto& n : shapes)
    for (int G : ghosts) {
      const int hg = G / 2;
      long long chunks = 0;
      for (int f = 0; f < 5; ++f) {
        const int sa = f >= F_VX ? f - F_VX : -1;
        std::set<std::tuple<int, int, int>> cover, want;
        for (int b = 0; b < 6; ++b) {
          const CuBox B = cu_box(n, G, sa, b);
          chunks += (long long)B.ez * B.ntx * B.nty;
          if (B.ez == 0) continue;
          if (B.tx < 1 || B.ty < 1 || B.tx > 64 || B.ty > 64 || B.tx * B.ty > kCuHosts) {
            std::printf("FAIL tile %dx%d n=%d,%d,%d G=%d\n", B.tx, B.ty, n[0], n[1], n[2], G);
            ++bad;
          }
          for (int pz = 0; pz < B.ez; ++pz)
            for (int ty = 0; ty < B.nty; ++ty)
              for (int tx = 0; tx < B.ntx; ++tx) {
                ++tiles;
                const int X0 = B.x0 + tx * B.tx, Y0 = B.y0 + ty * B.ty, h2 = B.z0 + pz;
                const int wx = B.x0 + B.ex - X0 < B.tx ? B.x0 + B.ex - X0 : B.tx;
                const int wy = B.y0 + B.ey - Y0 < B.ty ? B.y0 + B.ey - Y0 : B.ty;
                if (wx < 1 || wy < 1 || (wx + 2) * (wy + 2) > kCuZ || wy * (wx + 2) > kCuY) {
                  std::printf("FAIL width %d %d\n", wx, wy);
                  ++bad;
                }
                if (X0 - 1 < -hg - 1 || X0 + wx > (n[0] >> 1) + hg || Y0 - 1 < -hg - 1 ||
                    Y0 + wy > (n[1] >> 1) + hg || h2 - 1 < -hg - 1 || h2 + 1 > (n[2] >> 1) + hg) {
                  std::printf("FAIL halo at %d %d %d\n", X0, Y0, h2);
                  ++bad;
                }
                for (int y = Y0; y < Y0 + wy; ++y)
                  for (int x = X0; x < X0 + wx; ++x)
                    if (!cover.insert(std::make_tuple(x, y, h2)).second) {
                      std::printf("FAIL host %d %d %d twice\n", x, y, h2);
                      ++bad;
                    }
              }
        }
        // hosts with a ghost among their children: some axis where the host's two
        // children are not both kept (cells inside; for v_d faces strictly inside)
        for (int z = -hg; z < (n[2] >> 1) + hg; ++z)
          for (int y = -hg; y < (n[1] >> 1) + hg; ++y)
            for (int x = -hg; x < (n[0] >> 1) + hg; ++x) {
              const int h[3] = {x, y, z};
              bool kept = true;
              for (int a = 0; a < 3; ++a)
                kept = kept && h[a] >= (a == sa ? 1 : 0) && 2 * h[a] + 1 < n[a];
              if (!kept) want.insert(std::make_tuple(x, y, z));
            }
        if (cover != want) {
          std::printf("FAIL cover n=%d,%d,%d G=%d field %d: %zu vs %zu\n", n[0], n[1], n[2], G,
                      f, cover.size(), want.size());
          ++bad;
        }
      }
      if (chunks != cu_chunks(n, G)) {
        std::printf("FAIL chunks %lld vs %lld\n", chunks, cu_chunks(n, G));
        ++bad;
      }
    }
  if (bad) return 1;
  std::printf("OK %lld\n", tiles);
  return 0;
}
