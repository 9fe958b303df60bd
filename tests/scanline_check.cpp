// Host check of the SGM scanline tables (lfsgm_internal.cuh), built and run by test_scanlines.py.
// It prints the number of directions whose bit-field form (dir_of) differs from the table, then,
// for each (H, W) on the command line and each of the 16 directions r, it walks every scanline s
// from scan_start(r, s) for scan_steps pixels and prints one line
//   H W r n_scanlines covered twice missing bad_index bad_ends
// covered: pixels visited; twice: pixels visited more than once; missing: pixels never visited;
// bad_index: visited pixels whose scan_index is not s; bad_ends: scanlines whose start pixel's
// predecessor (p - r) or whose last pixel's successor (p + r) lies inside the image.
#include "lfsgm_internal.cuh"

#include <cstdio>
#include <cstdlib>
#include <vector>

using namespace lfsgm;

int main(int argc, char **argv) {
    // first line: directions whose bit-field form (dir_of) differs from the table
    int bad_dirs = 0;
    for (int r = 0; r < kMaxPaths; r++) {
        int dx, dy;
        dir_of(r, dx, dy);
        bad_dirs += dx != dir_dx(r) || dy != dir_dy(r);
    }
    printf("%d\n", bad_dirs);
    for (int a = 1; a + 1 < argc; a += 2) {
        const int H = atoi(argv[a]), W = atoi(argv[a + 1]);
        for (int r = 0; r < kMaxPaths; r++) {
            const int dx = dir_dx(r), dy = dir_dy(r);
            std::vector<int> seen((size_t)H * W, 0);
            long covered = 0, twice = 0, missing = 0, bad_index = 0, bad_ends = 0;
            const int ns = n_scanlines(r, H, W);
            auto inside = [&](int x, int y) { return x >= 0 && x < W && y >= 0 && y < H; };
            for (int s = 0; s < ns; s++) {
                int x, y;
                scan_start(r, s, H, W, x, y);
                const int len = scan_steps(x, y, dx, dy, H, W);
                if (inside(x - dx, y - dy) || inside(x + len * dx, y + len * dy) || len < 1) bad_ends++;
                for (int k = 0; k < len; k++) {
                    const int px = x + k * dx, py = y + k * dy;
                    if (!inside(px, py)) {
                        bad_ends++;
                        break;
                    }
                    covered++;
                    if (seen[(size_t)py * W + px]++) twice++;
                    if (scan_index(r, px, py, H, W) != s) bad_index++;
                }
            }
            for (int v : seen) missing += v == 0;
            printf("%d %d %d %d %ld %ld %ld %ld %ld\n", H, W, r, ns, covered, twice, missing, bad_index, bad_ends);
        }
    }
    return 0;
}
