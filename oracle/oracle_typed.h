/*
 * Typed body of the CPU oracle.  Included once per key type by ipm_oracle.c with
 *   T    the key type
 *   SUF  the name suffix (i32, u32, u64, f32)
 * defined.  TEST INFRASTRUCTURE ONLY (see the header of ipm_oracle.c).
 *
 * Every function is plain sequential C written from the paper's text:
 *   B. Bramas, Q. Bramas, "On the improvement of the in-place merge algorithm
 *   parallelization", arXiv 2005.12648.
 * Keys are only compared (with the type's own "<=") and moved, never computed.
 */

#define CAT2(a, b) a##_##b
#define CAT(a, b) CAT2(a, b)
#define FN(name) CAT(name, SUF)

/*
 * Stable merge, plain definition (Sec. 1, problem statement): the sorted array C of
 * size la+lb that contains A and B.  A tie takes the A element first, which is the
 * order std::inplace_merge gives (Sec. 4, the per-thread merge).
 */
void FN(orc_merge)(const T *a, uint64_t la, const T *b, uint64_t lb, T *out)
{
    uint64_t i = 0, j = 0;
    for (uint64_t t = 0; t < la + lb; ++t) {
        if (j == lb || (i < la && a[i] <= b[j]))
            out[t] = a[i++];
        else
            out[t] = b[j++];
    }
}

/* The same merge moving a 32-bit payload with each key (key-value form). */
void FN(orc_merge_kv)(const T *ka, const uint32_t *va, uint64_t la,
                      const T *kb, const uint32_t *vb, uint64_t lb,
                      T *kout, uint32_t *vout)
{
    uint64_t i = 0, j = 0;
    for (uint64_t t = 0; t < la + lb; ++t) {
        if (j == lb || (i < la && ka[i] <= kb[j])) {
            kout[t] = ka[i];
            vout[t] = va[i];
            ++i;
        } else {
            kout[t] = kb[j];
            vout[t] = vb[j];
            ++j;
        }
    }
}

/*
 * The same with a payload of w bytes per element (any record: it is only copied).
 */
void FN(orc_merge_kvw)(const T *ka, const unsigned char *va, uint64_t la,
                       const T *kb, const unsigned char *vb, uint64_t lb, uint64_t w,
                       T *kout, unsigned char *vout)
{
    uint64_t i = 0, j = 0;
    for (uint64_t t = 0; t < la + lb; ++t) {
        if (j == lb || (i < la && ka[i] <= kb[j])) {
            kout[t] = ka[i];
            memcpy(vout + t * w, va + i * w, (size_t)w);
            ++i;
        } else {
            kout[t] = kb[j];
            memcpy(vout + t * w, vb + j * w, (size_t)w);
            ++j;
        }
    }
}

/*
 * Exact split, first form: replay the plain merge and record, for each diagonal
 * d[k] (ascending, each <= la+lb), how many A elements are among the first d[k]
 * outputs.  This is the "optimal" split of Sec. 3.1 taken at a chosen output count.
 */
void FN(orc_splits_replay)(const T *a, uint64_t la, const T *b, uint64_t lb,
                           const uint64_t *d, uint64_t nd, uint64_t *out_i)
{
    uint64_t i = 0, j = 0, t = 0, k = 0;
    while (k < nd) {
        if (t == d[k]) {
            out_i[k++] = i;
            continue;
        }
        if (j == lb || (i < la && a[i] <= b[j]))
            ++i;
        else
            ++j;
        ++t;
    }
}

/*
 * Exact split, second (independent) form: binary search on the diagonal d for the
 * smallest m such that A[m] is not among the first d outputs.  A[m] is among them
 * exactly when A[m] <= B[d-1-m] (ties go to A).
 */
uint64_t FN(orc_split_bsearch)(const T *a, uint64_t la, const T *b, uint64_t lb, uint64_t d)
{
    uint64_t lo = d > lb ? d - lb : 0;
    uint64_t hi = d < la ? d : la;
    while (lo < hi) {
        uint64_t m = lo + (hi - lo) / 2;
        if (a[m] <= b[d - 1 - m])
            lo = m + 1;
        else
            hi = m;
    }
    return lo;
}

/*
 * Exact split by galloping from a guess (the correction step of the learned split
 * proposer, which has no counterpart in the paper): exponential steps 1, 2, 4, ...
 * away from the guess until the answer is bracketed, then bisection inside the
 * bracket.  *probes counts evaluations of the predicate.  The result equals
 * orc_split_bsearch for every guess.
 */
uint64_t FN(orc_gallop_split)(const T *a, uint64_t la, const T *b, uint64_t lb,
                              uint64_t d, uint64_t guess, uint64_t *probes)
{
    uint64_t lo = d > lb ? d - lb : 0;
    uint64_t hi = d < la ? d : la;
    uint64_t np = 0, L, R;
    if (guess < lo) guess = lo;
    if (guess > hi) guess = hi;
    /* pred(m): A[m] is among the first d outputs; true for m < answer. */
#define PRED(m) (++np, a[(m)] <= b[d - 1 - (m)])
    if (guess < hi && PRED(guess)) {
        /* answer in (guess, hi] */
        uint64_t prev = guess, step = 1;
        for (;;) {
            uint64_t m = guess + step;
            if (m >= hi) {
                L = prev + 1;
                R = hi;
                break;
            }
            if (PRED(m)) {
                prev = m;
                step *= 2;
            } else {
                L = prev + 1;
                R = m;
                break;
            }
        }
    } else {
        /* answer in [lo, guess] */
        uint64_t prev = guess, step = 1;
        for (;;) {
            if (guess < lo + step) {
                L = lo;
                R = prev;
                break;
            }
            uint64_t m = guess - step;
            if (!PRED(m)) {
                prev = m;
                step *= 2;
            } else {
                L = m + 1;
                R = prev;
                break;
            }
        }
    }
    while (L < R) {
        uint64_t m = L + (R - L) / 2;
        if (PRED(m))
            L = m + 1;
        else
            R = m;
    }
#undef PRED
    if (probes) *probes = np;
    return L;
}

/*
 * Linear shifting (Sec. 3.4, "Linear shifting (LS)"): exchange [X|Y] -> [Y|X] in
 * place.  The smaller block is swapped with the elements that occupy its final
 * place; it then stays untouched and the same problem remains on the rest.  When
 * X is on the left and is the smaller, its final place is the last |X| slots of Y
 * (the result is [Y_tail Y_head X]); when Y is the smaller, its final place is the
 * first |Y| slots of X (mirror case).  Equal blocks finish in one pairwise swap
 * (Sec. 3.5).  *nswaps counts elementary swaps.
 */
void FN(orc_ls_rotate)(T *p, uint64_t lx, uint64_t ly, uint64_t *nswaps)
{
    uint64_t ns = 0;
    while (lx > 0 && ly > 0) {
        if (lx <= ly) {
            T *q = p + ly; /* final place of X: the last lx slots */
            for (uint64_t t = 0; t < lx; ++t) {
                T tmp = p[t];
                p[t] = q[t];
                q[t] = tmp;
            }
            ns += lx;
            if (lx == ly) break;
            ly -= lx; /* rotate [Y_tail (lx) | Y_head (ly-lx)] at p */
        } else {
            T *q = p + lx; /* Y goes to the first ly slots */
            for (uint64_t t = 0; t < ly; ++t) {
                T tmp = p[t];
                p[t] = q[t];
                q[t] = tmp;
            }
            ns += ly;
            p += ly; /* rotate [X_tail (lx-ly) | X_head (ly)] at p+ly */
            lx -= ly;
        }
    }
    if (nswaps) *nswaps = ns;
}

/*
 * Circular shifting (Sec. 3.4, "Circular shifting" and its proof of correctness):
 * the element at index i of [A|B] goes to i+lb when i < la and to i-la otherwise.
 * Cycles start at indexes 0, 1, ..., t-1 with t = GCD(la, lb) (the proof's count;
 * the Background paragraph's "LCM cycles" contradicts it).  *ncycles and *nmoves
 * count cycles and element moves.
 */
void FN(orc_cs_rotate)(T *p, uint64_t la, uint64_t lb, uint64_t *ncycles, uint64_t *nmoves)
{
    uint64_t n = la + lb, moved = 0, cycles = 0;
    if (la != 0 && lb != 0) {
        for (uint64_t start = 0; moved < n; ++start) {
            T carry = p[start];
            uint64_t i = start;
            do {
                uint64_t dst = (i < la) ? i + lb : i - la;
                T tmp = p[dst];
                p[dst] = carry;
                carry = tmp;
                i = dst;
                ++moved;
            } while (i != start);
            ++cycles;
        }
    }
    if (ncycles) *ncycles = cycles;
    if (nmoves) *nmoves = moved;
}

/*
 * FindMedian (Alg. 1), read as follows where the listing is ambiguous: the two
 * midpoints are computed at the top of every iteration; when A[pA] == B[pB] that
 * pair is returned; otherwise the bounds move as the listing says; when a search
 * interval empties, the midpoints of the final intervals are returned.  The two
 * corner cases (A <= B, A > B) are tested first, as in the listing.
 */
void FN(orc_findmedian)(const T *a, uint64_t la, const T *b, uint64_t lb,
                        uint64_t *pa, uint64_t *pb)
{
    if (la == 0 || lb == 0 || a[la - 1] <= b[0]) {
        *pa = la;
        *pb = 0;
        return;
    }
    if (!(a[0] <= b[lb - 1])) {
        *pa = 0;
        *pb = lb;
        return;
    }
    uint64_t leftA = 0, limitA = la, leftB = 0, limitB = lb;
    while (leftA < limitA && leftB < limitB) {
        uint64_t mA = (limitA - leftA) / 2 + leftA;
        uint64_t mB = (limitB - leftB) / 2 + leftB;
        if (a[mA] == b[mB]) {
            *pa = mA;
            *pb = mB;
            return;
        }
        uint64_t A0 = mA, A1 = la - mA, B0 = mB, B1 = lb - mB;
        if (a[mA] < b[mB]) {
            if (A0 + B0 < A1 + B1)
                leftA = mA + 1;
            else
                limitB = mB;
        } else {
            if (A0 + B0 < A1 + B1)
                leftB = mB + 1;
            else
                limitA = mA;
        }
    }
    *pa = (limitA - leftA) / 2 + leftA;
    *pb = (limitB - leftB) / 2 + leftB;
}

/*
 * The sRecPar division strategy (Alg. 3), run sequentially: the task the master
 * creates for the right pair is executed as a recursive call, which gives the same
 * array because the two pairs are disjoint.  split_kind 0 uses the stable exact
 * split at the half diagonal, split_kind 1 uses FindMedian.  shift_kind 0 is linear
 * shifting, 1 circular shifting.  Pairs of at most size_limit elements, and the
 * pairs left at depth_limit, are merged with the plain stable merge through tmp
 * (which must hold size elements).  *moved_elems accumulates 2x the elementary
 * swaps of LS (each swap writes two slots) or the moves of CS.
 */
static void FN(srecpar_core)(T *arr, uint64_t start, uint64_t middle, uint64_t end,
                             int level, int depth_limit, uint64_t size_limit,
                             int split_kind, int shift_kind, T *tmp,
                             uint64_t *moved_elems)
{
    if (start == middle || middle == end) return;
    while (level != depth_limit && (end - start) > size_limit) {
        uint64_t la = middle - start, lb = end - middle, mA, mB;
        if (split_kind == 0) {
            uint64_t d = (end - start) / 2;
            mA = FN(orc_split_bsearch)(arr + start, la, arr + middle, lb, d);
            mB = d - mA;
        } else {
            FN(orc_findmedian)(arr + start, la, arr + middle, lb, &mA, &mB);
        }
        uint64_t restA = la - mA;
        if (shift_kind == 0) {
            uint64_t ns = 0;
            FN(orc_ls_rotate)(arr + start + mA, restA, mB, &ns);
            *moved_elems += 2 * ns;
        } else {
            uint64_t nc = 0, nm = 0;
            FN(orc_cs_rotate)(arr + start + mA, restA, mB, &nc, &nm);
            *moved_elems += nm;
        }
        FN(srecpar_core)(arr, start + mA + mB, start + mA + mB + restA, end,
                         level + 1, depth_limit, size_limit, split_kind, shift_kind,
                         tmp, moved_elems);
        end = start + mA + mB;
        middle = start + mA;
        ++level;
        if (start == middle || middle == end) return;
    }
    FN(orc_merge)(arr + start, middle - start, arr + middle, end - middle, tmp);
    memcpy(arr + start, tmp, (size_t)(end - start) * sizeof(T));
}

void FN(orc_srecpar)(T *arr, uint64_t middle, uint64_t size, int depth_limit,
                     uint64_t size_limit, int split_kind, int shift_kind, T *tmp,
                     uint64_t *moved_elems)
{
    uint64_t mv = 0;
    if (!(middle == 0 || middle == size || arr[middle - 1] <= arr[middle]))
        FN(srecpar_core)(arr, 0, middle, size, 0, depth_limit, size_limit, split_kind,
                         shift_kind, tmp, &mv);
    if (moved_elems) *moved_elems = mv;
}

/*
 * The division of Alg. 3 without the data movement (the pair boundaries its recursion
 * reaches), for the balance comparison of Sec. 4 (FindMedian against the optimal
 * split).  Level by level, every region [A[ia[k0], ia[k1]) | B[jb[k0], jb[k1])) is cut
 * in two at its pivot (pA, pB): the exact stable split at the region's half diagonal
 * floor(c/2) (split_kind 0) or FindMedian (split_kind 1).  A region with an empty side
 * is not divided further, as in Alg. 3 (it needs no merge); it stays whole in its left
 * child and its right child is empty.  Outputs the 2^depth + 1 boundaries:
 * pair k = A[ia[k], ia[k+1]) with B[jb[k], jb[k+1]).
 */
void FN(orc_division)(const T *a, uint64_t la, const T *b, uint64_t lb, int depth,
                      int split_kind, uint64_t *ia, uint64_t *jb)
{
    const uint64_t P = (uint64_t)1 << depth;
    ia[0] = 0;
    jb[0] = 0;
    ia[P] = la;
    jb[P] = lb;
    for (int l = 0; l < depth; ++l) {
        const uint64_t step = P >> l;
        for (uint64_t k0 = 0; k0 < P; k0 += step) {
            const uint64_t k1 = k0 + step, mid = k0 + step / 2;
            const uint64_t ra = ia[k1] - ia[k0], rb = jb[k1] - jb[k0];
            uint64_t pa, pb;
            if (ra == 0 || rb == 0) {
                pa = ra;
                pb = rb;
            } else if (split_kind == 0) {
                const uint64_t d = (ra + rb) / 2;
                pa = FN(orc_split_bsearch)(a + ia[k0], ra, b + jb[k0], rb, d);
                pb = d - pa;
            } else {
                FN(orc_findmedian)(a + ia[k0], ra, b + jb[k0], rb, &pa, &pb);
            }
            ia[mid] = ia[k0] + pa;
            jb[mid] = jb[k0] + pb;
        }
    }
}

/*
 * The layout the division stage produces (Sec. 3): A_0 B_0 A_1 B_1 ... A_{P-1}
 * B_{P-1}, where pair k holds A[i_k, i_{k+1}) and B[j_k, j_{k+1}) with
 * j_k = d_k - i_k.  Written out of place from the split table (d, i), P+1 entries.
 */
void FN(orc_arrange)(const T *a, uint64_t la, const T *b, uint64_t lb,
                     const uint64_t *d, const uint64_t *i, uint64_t P, T *out)
{
    (void)la;
    (void)lb;
    for (uint64_t k = 0; k < P; ++k) {
        uint64_t i0 = i[k], i1 = i[k + 1];
        uint64_t j0 = d[k] - i0, j1 = d[k + 1] - i1;
        T *o = out + d[k];
        for (uint64_t t = i0; t < i1; ++t) *o++ = a[t];
        for (uint64_t t = j0; t < j1; ++t) *o++ = b[t];
    }
}

#undef FN
#undef CAT
#undef CAT2
