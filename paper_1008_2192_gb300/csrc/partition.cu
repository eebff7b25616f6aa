// The paper's 2-D image segmentation (declaration and contract in
// include/crb.h): a frame cut into cols x rows rectangles of nearly equal
// area, each widened by a context margin on every side that touches another
// rectangle. CRBLASTER hands each such sub-image to one actor (Sec. 6.2); its
// 2-D algorithm takes the factorisation of N that makes the sub-images closest
// to square, so that a prime N falls back to 1 x N horizontal slices, the
// older 1-D scheme (Sec. 6.3.1, Sec. 7). Host code only.

#include <cmath>
#include <string>

#include "crb.h"

void crb_detail_set_error(const char* msg);  // crb.cu

namespace {

// How far the sub-images of a cols x rows cut of a w x h frame are from square.
double squareness(int w, int h, int cols, int rows) {
  return std::fabs(std::log((double(w) / cols) / (double(h) / rows)));
}

// Start of part i of n parts of len (the first len % n parts one longer).
int part_start(int len, int n, int i) {
  const int base = len / n, extra = len % n;
  return i * base + (i < extra ? i : extra);
}

}  // namespace

extern "C" int crb_partition(int w, int h, int nparts, int cols, int context, crb_rect* rects, int max_rects,
                             int* out_cols, int* out_rows) {
  if (w < 1 || h < 1 || nparts < 1 || cols < 0 || context < 0) {
    crb_detail_set_error("crb_partition: need w, h, nparts >= 1, cols >= 0, context >= 0");
    return -CRB_EINVAL;
  }
  int best_c = 0;
  if (cols > 0) {
    if (nparts % cols != 0 || cols > w || nparts / cols > h) {
      crb_detail_set_error("crb_partition: cols must divide nparts, with cols <= w and nparts / cols <= h");
      return -CRB_EINVAL;
    }
    best_c = cols;
  } else {
    double best = 0;
    for (int c = 1; c <= nparts; ++c) {  // ascending: a tie keeps the fewer columns
      if (nparts % c != 0 || c > w || nparts / c > h) continue;
      const double q = squareness(w, h, c, nparts / c);
      if (best_c == 0 || q < best - 1e-12) {
        best = q;
        best_c = c;
      }
    }
    if (best_c == 0) {
      crb_detail_set_error("crb_partition: no cols x rows = nparts cut fits the frame");
      return -CRB_EINVAL;
    }
  }
  if (context > w || context > h) context = w > h ? w : h;  // no wider than the frame (and no overflow below)
  const int best_r = nparts / best_c;
  if (out_cols) *out_cols = best_c;
  if (out_rows) *out_rows = best_r;
  if (!rects || max_rects < nparts) return nparts;
  for (int r = 0; r < best_r; ++r)
    for (int c = 0; c < best_c; ++c) {
      crb_rect& o = rects[r * best_c + c];
      o.x0 = part_start(w, best_c, c);
      o.y0 = part_start(h, best_r, r);
      o.w = part_start(w, best_c, c + 1) - o.x0;
      o.h = part_start(h, best_r, r + 1) - o.y0;
      o.cx0 = o.x0 - context > 0 ? o.x0 - context : 0;
      o.cy0 = o.y0 - context > 0 ? o.y0 - context : 0;
      const int cx1 = o.x0 + o.w + context < w ? o.x0 + o.w + context : w;
      const int cy1 = o.y0 + o.h + context < h ? o.y0 + o.h + context : h;
      o.cw = cx1 - o.cx0;
      o.ch = cy1 - o.cy0;
    }
  return nparts;
}
