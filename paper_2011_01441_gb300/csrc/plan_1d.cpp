// PACO 1D partition (Sec. "PACO 1D"): the work of Eq. (1D) is the triangle
// {(i, j): 0 <= i < j <= n}.  The cache-oblivious recursion on an output
// range [lo, hi) runs the left half's triangle, then the square that
// updates the right half's outputs from the left half's inputs, then the
// right half's triangle.  PACO changes only how each square is run on p
// processors: the square (with the list of all p processors) is cut along
// its longer side into two parts in the ratio floor(p/2) : ceil(p/2), the
// processor list is split the same way, and each part recurses with its
// list until a rectangle owns one processor.  A cut along the input side
// makes the two parts update the same outputs, so the second part works in
// temporary space that is merged (a min) into the outputs after the phase.
// Triangles at most `base` wide are base cases run on one processor.
#include "../../include/paco_plan.h"

#include <cstdint>
#include <vector>

namespace {

struct Builder {
    int p;
    int64_t base;
    int32_t phase = 0;
    int32_t groups = 0;
    int64_t temp = 0;
    std::vector<paco_1d_task> tasks;

    void emit(int64_t j0, int64_t j1, int64_t i0, int64_t i1, int32_t proc, int32_t kind, int32_t group) {
        paco_1d_task t;
        t.j0 = j0;
        t.j1 = j1;
        t.i0 = i0;
        t.i1 = i1;
        t.proc = proc;
        t.phase = phase;
        t.merge_group = group;
        t.kind = kind;
        tasks.push_back(t);
    }

    // rectangle: outputs [j0, j1) x inputs [i0, i1), processors [q0, q0 + q)
    void square(int64_t j0, int64_t j1, int64_t i0, int64_t i1, int q0, int q, int32_t group) {
        if (q == 1 || (j1 - j0 <= 1 && i1 - i0 <= 1)) {
            emit(j0, j1, i0, i1, q0, 1, group);
            return;
        }
        const int k = q / 2;
        const int64_t w = j1 - j0, h = i1 - i0;
        if (w >= h) {   // cut the output side (ties: no temporary space needed)
            const int64_t w1 = w * k / q;
            square(j0, j0 + w1, i0, i1, q0, k, group);
            square(j0 + w1, j1, i0, i1, q0 + k, q - k, group);
        } else {        // cut the input side: the second part writes temporary space
            const int64_t h1 = h * k / q;
            square(j0, j1, i0, i0 + h1, q0, k, group);
            const int32_t g = groups++;
            temp += w;
            square(j0, j1, i0 + h1, i1, q0 + k, q - k, g);
        }
    }

    void solve(int64_t lo, int64_t hi) {
        if (hi - lo <= base) {
            emit(lo, hi, lo, hi, 0, 0, -1);
            ++phase;
            return;
        }
        const int64_t mid = lo + (hi - lo) / 2;
        solve(lo, mid);
        square(mid, hi, lo, mid, 0, p, -1);
        ++phase;
        solve(mid, hi);
    }
};

}  // namespace

extern "C" int paco_plan_1d(int64_t n, int32_t p, int64_t base, paco_1d_task *out, int64_t cap, int64_t *count,
                            int32_t *phases, int64_t *temp_words) {
    if (n < 0 || p < 1 || base < 1) return -1;
    Builder B;
    B.p = p;
    B.base = base;
    B.solve(0, n + 1);
    if (count) *count = (int64_t)B.tasks.size();
    if (phases) *phases = B.phase;
    if (temp_words) *temp_words = B.temp;
    for (int64_t k = 0; out && k < (int64_t)B.tasks.size() && k < cap; ++k) out[k] = B.tasks[(size_t)k];
    return 0;
}
