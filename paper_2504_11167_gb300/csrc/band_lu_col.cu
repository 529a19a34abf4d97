// Banded LU of every partition A_i, column by column (no pivoting; the
// D-stage factorisation of paper section 2.1, "A = D S", with each A_i
// factorised on its own).  It produces the packed solve tiles of the
// block-recursive kernel in factor_lu.cu, with the same values up to rounding:
//   LT[J] = [ L_JJ^{-1} strictly lower | L_{J,J-1} upper incl. diagonal ]
//   UT[J] = [ (D^{-1}U_JJ)^{-1} strictly upper | D^{-1}U_{J,J+1} lower incl. diagonal ]
//   DI[J] = D^{-1},  D = diag(U_JJ)
// in two kernels.
//
// k_band_lu_col: one CTA per partition eliminates its columns, TR at a time.
//   Without pivoting, eliminating column j changes only rows and columns
//   j+1..j+k, so the live part of the matrix is a KB x KB window (KB >= k)
//   that slides down the diagonal.  The window stays in registers, indexed
//   modulo KB: entry (i, l) sits with the thread owning row residue i mod KB
//   and column residue l mod KB (a GRID x GRID thread grid, TR x TR residues
//   per thread).  One step eliminates the TR columns j..j+TR-1 of one residue
//   group (one barrier per step):
//     - the pivot block a_{j+u, j+v}, the pivot rows and the pivot columns
//       were published by their owners in shared memory (double-buffered);
//     - every thread factors the TR x TR pivot block itself (P = L_p U_p);
//     - every thread forms the pivot-row entries L_p^{-1} R of its columns and
//       the multipliers C U_p^{-1} of its rows;
//     - the thread row / column owning the group's residues swaps in the
//       entering rows and columns j+KB..j+KB+TR-1 (straight from the band: no
//       earlier column touches them);
//     - every thread applies the rank-TR update to its TR x TR entries;
//     - the owners of the next group publish it.
//   The leaving residue slots stand for the entering columns in the pivot
//   rows and for the entering rows in the pivot columns.  Those "far" entries
//   come from the band as well.
//   Staging is spread evenly over all threads.  Each thread owns the same few
//   values in every group, each a fixed band diagonal with a precomputed
//   pointer.  Per step it:
//     - issues 8-byte cp.async for the group PD steps ahead (32 columns);
//     - converts its own values of the next group to the working precision,
//       in integer arithmetic (d2f_rn: GB300's hardware FP64 conversion runs
//       on the slow FP64 units);
//     - writes its share of the previous block's multipliers.
//   Outputs:
//     - the multipliers of a block's KB columns are staged in shared memory
//       and written during the next block;
//     - pivot row j scaled by 1/u_jj is row j mod KB of UT;
//     - DI = 1/u_jj.
//   At that point LT and UT hold L_JJ and D^{-1}U_JJ themselves in their
//   strict triangles.
// k_band_lu_inv: for every block (all independent) inverts those two unit
//   lower triangular matrices in place (D^{-1}U_JJ after reversing its rows
//   and columns: with P the reversal, P U P is lower triangular and
//   (P U P)^{-1} = P U^{-1} P).  In halves H = KB/2:
//     X11 = M11^{-1}, X22 = M22^{-1}   one thread per column (forward
//                                      substitution, the column in registers);
//     X21 = -X22 (M21 X11)             4 x 4 register-tiled products;
//   all in one shared-memory copy of the two matrices.
#include "common.cuh"
#include "internal.h"
#include "tile_ops.cuh"

namespace lrs {

template <typename T, int KB> struct ColGeo {
    static constexpr int GRID = KB >= 16 ? 16 : 8;    // thread grid GRID x GRID
    static constexpr int NT = GRID * GRID;
    static constexpr int TR = KB / GRID;              // residues per thread and direction; columns per step
    static constexpr int PD = (sizeof(T) == 8 ? 16 : 32) / TR;  // staging distance in steps
    static constexpr int RING = PD + 1;               // raw ring slots (step Gs in slot Gs % RING)
    static constexpr int SLOT = 2 * TR * KB + 2 * TR * TR;  // staged values per step
    static constexpr int SLOTP = (SLOT + 3) / 4 * 4;  // converted stride (16-byte aligned vectors)
    static constexpr int PUB = TR * TR + 2 * TR * KB; // published values per step
    static constexpr int NU = (SLOT + NT - 1) / NT;   // staged values per thread and step
};

template <typename T, int KB> struct ColSmem {
    using G = ColGeo<T, KB>;
    static constexpr int LDL = KB + 16 / (int)sizeof(T);  // multiplier staging row stride
    static constexpr size_t bytes = (size_t)G::RING * G::SLOT * 8 + (size_t)2 * G::SLOTP * sizeof(T) +
                                    (size_t)2 * G::PUB * sizeof(T) + (size_t)2 * KB * LDL * sizeof(T);
};

template <typename T, int KB>
__global__ void __launch_bounds__(ColGeo<T, KB>::NT, sizeof(T) == 4 ? 2 : 1)
    k_band_lu_col(const double *__restrict__ band, int64_t ld, int k, Parts P, T *__restrict__ LT,
                  T *__restrict__ UT, T *__restrict__ DI, int64_t *__restrict__ status) {
    using G = ColGeo<T, KB>;
    constexpr int GRID = G::GRID, NT = G::NT, TR = G::TR, PD = G::PD, RING = G::RING, SLOT = G::SLOT,
                  SLOTP = G::SLOTP, PUB = G::PUB, NU = G::NU;
    constexpr int LDL = ColSmem<T, KB>::LDL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *raw = reinterpret_cast<double *>(smem_raw);  // [RING][SLOT] staged band values
    T *cv_ = reinterpret_cast<T *>(raw + RING * SLOT);   // [2][SLOTP] converted, by step parity:
    //   ER [TR][KB] entering rows by column residue, EC [TR][KB] entering columns by row residue,
    //   FR [TR][TR] far pivot-row entries, FC [TR][TR] far pivot-column entries (of the next step)
    T *pub = cv_ + 2 * SLOTP;                            // [2][PUB] published, by step parity:
    //   PB [TR][TR] pivot block, RB [TR][KB] pivot rows by column residue, CB [TR][KB] pivot columns by row residue
    T *LS = pub + 2 * PUB;                               // [2][KB][LDL] multipliers [column][row residue]

    const int part = blockIdx.x;
    const int64_t s0 = P.off[part], ni = P.off[part + 1] - s0, b0 = P.boff[part];
    const int nb = (int)(P.boff[part + 1] - b0);
    const int NP = nb * KB;  // padded columns of the partition
    const int NG = nb * GRID;
    const int t = threadIdx.x, ty = t / GRID, tx = t % GRID;

    // partition-local entry, identity beyond the partition
    auto entry = [&](int64_t i, int64_t l) -> double {
        if (i >= ni || l >= ni) return (i == l) ? 1.0 : 0.0;
        const int64_t d = k + i - l;
        return (d < 0 || d > 2 * k) ? 0.0 : band[d * ld + s0 + l];
    };
    // Thread t stages slots e = t + u NT of every step; slot e of the step at
    // column jb is entry(jb + iofs, jb + lofs), one band diagonal:
    //   e < TR KB:    entering row jb+KB+v at column jb+KB+TR-1-o    (v = e / KB, o = e % KB)
    //   e < 2 TR KB:  entering column jb+KB+v at row jb+KB+TR-1-o
    //   next:         far pivot-row entry a_{jb+TR+u, jb+TR+KB+v}   (u, v < TR)
    //   last:         far pivot-column entry a_{jb+TR+KB+v, jb+TR+u}
    // The entering values go to the residue (jb + TR-1-o) mod KB.
    const double *src[NU];
    int so[NU], rofs[NU], hi_ofs[NU];
    bool live[NU], inb[NU], idn[NU];
    // The partial last round of slots (REM of them) goes to the last REM
    // threads, so that the extra staging and conversion do not fall on the
    // first warp (the per-step outputs rotate over the warps too, below).
    constexpr int REM = SLOT - (NU - 1) * NT;  // slots of the last round (1..NT)
#pragma unroll
    for (int u = 0; u < NU; ++u) {
        const int e = (u == NU - 1) ? (u * NT + t - (NT - REM)) : (t + u * NT);
        live[u] = (u == NU - 1) ? (t >= NT - REM) : (e < SLOT);
        so[u] = e;
        int iofs, lofs;
        rofs[u] = 0;
        if (e < TR * KB) {
            const int v = e / KB, o = e % KB;
            iofs = KB + v; lofs = KB + TR - 1 - o; rofs[u] = TR - 1 - o;
        } else if (e < 2 * TR * KB) {
            const int v = (e - TR * KB) / KB, o = (e - TR * KB) % KB;
            iofs = KB + TR - 1 - o; lofs = KB + v; rofs[u] = TR - 1 - o;
        } else if (e < 2 * TR * KB + TR * TR) {
            const int uu = (e - 2 * TR * KB) / TR, v = (e - 2 * TR * KB) % TR;
            iofs = TR + uu; lofs = TR + KB + v;
        } else {
            const int uu = (e - 2 * TR * KB - TR * TR) / TR, v = (e - 2 * TR * KB - TR * TR) % TR;
            iofs = TR + KB + v; lofs = TR + uu;
        }
        if (!live[u]) { iofs = 0; lofs = 0; }
        const int dg = k + iofs - lofs;
        inb[u] = live[u] && dg >= 0 && dg <= 2 * k;
        src[u] = band + s0 + lofs + (inb[u] ? (int64_t)dg * ld : 0);
        hi_ofs[u] = iofs > lofs ? iofs : lofs;  // beyond the partition once jb + hi_ofs >= ni
        idn[u] = iofs == lofs;
    }
    auto stage = [&](int Gs) {
        double *r = raw + (Gs % RING) * SLOT;
        const int jb = Gs * TR;
#pragma unroll
        for (int u = 0; u < NU; ++u) {
            if (!live[u]) continue;
            if (inb[u] && jb + hi_ofs[u] < ni) cp_async_small<8>(r + so[u], src[u] + jb);
            else r[so[u]] = (jb + hi_ofs[u] >= ni && idn[u]) ? 1.0 : 0.0;
        }
    };
    auto convert = [&](int Gs) {
        const double *r = raw + (Gs % RING) * SLOT;
        T *c = cv_ + (Gs & 1) * SLOTP;
        const int jb = Gs * TR;
#pragma unroll
        for (int u = 0; u < NU; ++u) {
            if (!live[u]) continue;
            const int e = so[u];
            int pos = e;  // far entries keep their slot
            if (e < 2 * TR * KB) pos = (e / KB) * KB + ((jb + rofs[u]) & (KB - 1));
            c[pos] = from_f64<T>(r[e]);
        }
    };

    // window of columns 0..KB-1; published pivot block, rows and columns of step 0
    T w[TR][TR];
#pragma unroll
    for (int r = 0; r < TR; ++r)
#pragma unroll
        for (int c = 0; c < TR; ++c) w[r][c] = (T)entry(ty * TR + r, tx * TR + c);
    for (int e = t; e < PUB; e += NT) {
        T v;
        if (e < TR * TR) v = (T)entry(e / TR, e % TR);
        else if (e < TR * TR + TR * KB) {
            const int u = (e - TR * TR) / KB, gm = (e - TR * TR) % KB;
            v = (T)(gm < TR ? entry(u, KB + gm) : entry(u, gm));
        } else {
            const int u = (e - TR * TR - TR * KB) / KB, rh = (e - TR * TR - TR * KB) % KB;
            v = (T)(rh < TR ? entry(KB + rh, u) : entry(rh, u));
        }
        pub[e] = v;
    }
    for (int e = t; e < KB * KB; e += NT)  // no L_{0,-1}
        if (e / KB <= e % KB) LT[b0 * KB * KB + e] = T(0);
    for (int Gs = 0; Gs < PD; ++Gs) {
        if (Gs < NG) stage(Gs);
        cp_async_commit();
    }
    cp_async_wait<PD - 1>();
    convert(0);

    for (int Gi = 0; Gi < NG; ++Gi) {
        const int g = Gi % GRID, J = Gi / GRID, j = Gi * TR;
        const bool rowg = (ty == g), colg = (tx == g);
        __syncthreads();
        // ring slot of step Gi-1 (converted during step Gi-2); step Gi+1 into the other parity
        if (Gi + PD < NG) stage(Gi + PD);
        cp_async_commit();
        cp_async_wait<PD - 1>();
        if (Gi + 1 < NG) convert(Gi + 1);
        if (J > 0) {  // tile rows g*TR.. of the previous block's multipliers
            const T *ls = LS + ((J - 1) & 1) * KB * LDL;
            T *lt = LT + (b0 + J - 1) * KB * KB;
            for (int e = t; e < TR * KB; e += NT) {
                const int a2 = g * TR + e / KB, b = e % KB;
                lt[(a2 > b ? 0 : KB * KB) + a2 * KB + b] = ls[b * LDL + a2];
            }
        }
        const T *PB = pub + (Gi & 1) * PUB, *RB = PB + TR * TR, *CB = RB + TR * KB;
        const T *cg = cv_ + (Gi & 1) * SLOTP;
        // pivot block P = L_p U_p (every thread; U_p in place, unit L_p below it)
        T pv[TR][TR], pinv[TR];
#pragma unroll
        for (int u = 0; u < TR; ++u) ld_row<T, TR>(PB + u * TR, pv[u]);
#pragma unroll
        for (int p = 0; p < TR; ++p) {
            if (t == 0 && !usable_pivot<T>(pv[p][p]))
                atomicMin((unsigned long long *)status, (unsigned long long)(s0 + j + p));
            pinv[p] = fast_rcp<T>(pv[p][p]);
#pragma unroll
            for (int q = p + 1; q < TR; ++q) {
                const T l = pv[q][p] * pinv[p];
                pv[q][p] = l;
#pragma unroll
                for (int c = p + 1; c < TR; ++c) pv[q][c] -= l * pv[p][c];
            }
        }
        // pivot-row entries of my columns: L_p^{-1} R;  multipliers of my rows: C U_p^{-1}
        T ur[TR][TR], m[TR][TR];  // ur[u][c], m[r][u]
#pragma unroll
        for (int u = 0; u < TR; ++u) {
            ld_row<T, TR>(RB + u * KB + tx * TR, ur[u]);
#pragma unroll
            for (int p = 0; p < u; ++p) {
                if constexpr (sizeof(T) == 4 && TR % 2 == 0) {
                    const float2 nl = make_float2(-pv[u][p], -pv[u][p]);
#pragma unroll
                    for (int c = 0; c < TR; c += 2) {
                        const float2 o = __ffma2_rn(nl, make_float2(ur[p][c], ur[p][c + 1]),
                                                    make_float2(ur[u][c], ur[u][c + 1]));
                        ur[u][c] = o.x;
                        ur[u][c + 1] = o.y;
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < TR; ++c) ur[u][c] -= pv[u][p] * ur[p][c];
                }
            }
        }
        {
            T cb[TR][TR];  // cb[u][r]
#pragma unroll
            for (int u = 0; u < TR; ++u) ld_row<T, TR>(CB + u * KB + ty * TR, cb[u]);
#pragma unroll
            for (int r = 0; r < TR; ++r)
#pragma unroll
                for (int u = 0; u < TR; ++u) {
                    T y = cb[u][r];
#pragma unroll
                    for (int p = 0; p < u; ++p) y -= m[r][p] * pv[p][u];
                    m[r][u] = y * pinv[u];
                }
        }
        // rows and columns j..j+TR-1 leave; rows and columns j+KB.. enter
        if (rowg) {
#pragma unroll
            for (int v = 0; v < TR; ++v) ld_row<T, TR>(cg + v * KB + tx * TR, w[v]);
        }
        if (colg) {
#pragma unroll
            for (int v = 0; v < TR; ++v) {
                T ec[TR];
                ld_row<T, TR>(cg + TR * KB + v * KB + ty * TR, ec);
#pragma unroll
                for (int r = 0; r < TR; ++r) w[r][v] = ec[r];
            }
        }
        if constexpr (sizeof(T) == 4 && TR % 2 == 0) {
            // two columns per packed FP32 FMA: each half of __ffma2_rn rounds
            // like fmaf, so the window holds the values of the scalar form
#pragma unroll
            for (int u = 0; u < TR; ++u)
#pragma unroll
                for (int r = 0; r < TR; ++r) {
                    const float2 nm = make_float2(-m[r][u], -m[r][u]);
#pragma unroll
                    for (int c = 0; c < TR; c += 2) {
                        const float2 o = __ffma2_rn(nm, make_float2(ur[u][c], ur[u][c + 1]),
                                                    make_float2(w[r][c], w[r][c + 1]));
                        w[r][c] = o.x;
                        w[r][c + 1] = o.y;
                    }
                }
        } else {
#pragma unroll
            for (int u = 0; u < TR; ++u)
#pragma unroll
                for (int r = 0; r < TR; ++r)
#pragma unroll
                    for (int c = 0; c < TR; ++c) w[r][c] -= m[r][u] * ur[u][c];
        }
        // outputs: multipliers (staged), scaled pivot rows, 1/u_jj; in the leaving
        // slots the pivot block's own L_p (below) and U_p (above) entries
        if (tx == 0) {
            T *ls = LS + (J & 1) * KB * LDL;
#pragma unroll
            for (int u = 0; u < TR; ++u) {
                T v[TR];
#pragma unroll
                for (int r = 0; r < TR; ++r) v[r] = (rowg && r > u) ? pv[r][u] : m[r][u];
                st_row<T, TR>(ls + (g * TR + u) * LDL + ty * TR, v);
            }
        }
        // scaled pivot rows: every thread row holds them; row (g + GRID/2) mod GRID
        // writes them, so the work moves from warp to warp
        const int tw = (g + GRID / 2) % GRID;
        if (ty == tw) {
            T *ut = UT + ((b0 + J) * KB + g * TR) * KB + tx * TR;
#pragma unroll
            for (int u = 0; u < TR; ++u) {
                T v[TR];
#pragma unroll
                for (int c = 0; c < TR; ++c) v[c] = ((colg && c > u) ? pv[u][c] : ur[u][c]) * pinv[u];
                st_row<T, TR>(ut + u * KB, v);
            }
        }
        if (ty == tw && tx == 0) {
#pragma unroll
            for (int u = 0; u < TR; ++u) DI[b0 * KB + j + u] = pinv[u];
        }
        // publish the next step
        if (j + TR < NP) {
            const int g1 = (g + 1) % GRID;
            T *PB1 = pub + ((Gi + 1) & 1) * PUB, *RB1 = PB1 + TR * TR, *CB1 = RB1 + TR * KB;
            if (ty == g1 && tx == g1) {
#pragma unroll
                for (int u = 0; u < TR; ++u) {
                    st_row<T, TR>(PB1 + u * TR, w[u]);
                    T fr[TR], fc[TR];
                    ld_row<T, TR>(cg + 2 * TR * KB + u * TR, fr);
                    ld_row<T, TR>(cg + 2 * TR * KB + TR * TR + u * TR, fc);
                    st_row<T, TR>(RB1 + u * KB + g1 * TR, fr);
                    st_row<T, TR>(CB1 + u * KB + g1 * TR, fc);
                }
            } else if (ty == g1) {
#pragma unroll
                for (int u = 0; u < TR; ++u) st_row<T, TR>(RB1 + u * KB + tx * TR, w[u]);
            } else if (tx == g1) {
#pragma unroll
                for (int u = 0; u < TR; ++u) {
                    T v[TR];
#pragma unroll
                    for (int r = 0; r < TR; ++r) v[r] = w[r][u];
                    st_row<T, TR>(CB1 + u * KB + ty * TR, v);
                }
            }
        }
    }
    __syncthreads();
    // multipliers of the last block (no block below it)
    for (int e = t; e < KB * KB; e += NT) {
        const int a = e / KB, b = e % KB;
        if (a > b) LT[(b0 + nb - 1) * KB * KB + e] = LS[((nb - 1) & 1) * KB * LDL + b * LDL + a];
    }
}

// The same factorisation one column per step (FP64: the TR-column step's
// registers (pivot block, pivot-row entries and multipliers in doubles) would
// leave room for only one CTA per SM).  Per column: one barrier; the owners of
// pivot row and column j+1 publish them after the rank-1 update; staging,
// conversion and flushing are spread over the columns of each group of TR.
template <typename T, int KB> struct Col1Geo {
    static constexpr int GRID = KB >= 16 ? 16 : 8;   // thread grid GRID x GRID
    static constexpr int NT = GRID * GRID;
    static constexpr int TR = KB / GRID;             // residues per thread and direction; columns per group
    static constexpr int PD = 32 / TR;               // staging distance in groups (32 columns)
    static constexpr int RING = PD + 1;              // raw ring slots (group Gs in slot Gs % RING)
    static constexpr int CW = 2 * KB + 2;            // staged values per column
    static constexpr int CWP = (CW + 3) / 4 * 4;     // converted row stride (16-byte aligned vectors)
    static constexpr int SLOT = TR * CW;             // staged values per group
    static constexpr int NU = (SLOT + NT - 1) / NT;  // staged values per thread and group
};

template <typename T, int KB> struct Col1Smem {
    using G = Col1Geo<T, KB>;
    static constexpr int LDL = KB + 16 / (int)sizeof(T);  // multiplier staging row stride
    static constexpr size_t raw = (size_t)G::RING * G::SLOT * 8;
    static constexpr size_t cvt = (size_t)2 * G::TR * G::CWP * sizeof(T);
    static constexpr size_t bytes = raw + cvt + (size_t)4 * KB * sizeof(T) + 16 + (size_t)2 * KB * LDL * sizeof(T);
};

template <typename T, int KB>
__global__ void __launch_bounds__(Col1Geo<T, KB>::NT)
    k_band_lu_col1(const double *__restrict__ band, int64_t ld, int k, Parts P, T *__restrict__ LT,
                  T *__restrict__ UT, T *__restrict__ DI, int64_t *__restrict__ status) {
    using G = Col1Geo<T, KB>;
    constexpr int GRID = G::GRID, NT = G::NT, TR = G::TR, PD = G::PD, RING = G::RING, CW = G::CW,
                  CWP = G::CWP, SLOT = G::SLOT, NU = G::NU;
    constexpr int LDL = Col1Smem<T, KB>::LDL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *raw = reinterpret_cast<double *>(smem_raw);  // [RING][SLOT] staged band values
    T *cv_ = reinterpret_cast<T *>(raw + RING * SLOT);   // [2][TR][CWP] converted, by group parity:
                                                         //   [0, KB) entering row by column residue,
                                                         //   [KB, 2KB) entering column by row residue,
                                                         //   2KB, 2KB+1: far ends of the next pivot row / column
    T *rowb = cv_ + 2 * TR * CWP;                        // [2][KB] pivot row, by column residue
    T *colb = rowb + 2 * KB;                             // [2][KB] pivot column, by row residue
    T *pivb = colb + 2 * KB;                             // [2] pivots (16 bytes reserved)
    T *LS = pivb + 16 / sizeof(T);                       // [2][KB][LDL] multipliers [column][row residue]

    const int part = blockIdx.x;
    const int64_t s0 = P.off[part], ni = P.off[part + 1] - s0, b0 = P.boff[part];
    const int nb = (int)(P.boff[part + 1] - b0);
    const int NP = nb * KB;  // padded columns of the partition
    const int NG = nb * GRID;
    const int t = threadIdx.x, ty = t / GRID, tx = t % GRID;

    // partition-local entry, identity beyond the partition
    auto entry = [&](int64_t i, int64_t l) -> double {
        if (i >= ni || l >= ni) return (i == l) ? 1.0 : 0.0;
        const int64_t d = k + i - l;
        return (d < 0 || d > 2 * k) ? 0.0 : band[d * ld + s0 + l];
    };
    // Thread t stages slots e = t + u NT of every group: column s = e / CW of
    // the group, value o = e % CW, which is entry(jj + iofs, jj + lofs) for
    // the group's column jj:
    //   o < KB:  (jj+KB, jj+KB-o)       o < 2KB: (jj+KB-o', jj+KB), o' = o-KB
    //   2KB:     (jj+1, jj+1+KB)        2KB+1:   (jj+1+KB, jj+1)
    // i.e. one band diagonal at column jj + lofs.
    const double *src[NU];
    int sc[NU], so[NU], hi_ofs[NU];
    bool live[NU], inb[NU], idn[NU];
#pragma unroll
    for (int u = 0; u < NU; ++u) {
        const int e = t + u * NT;
        live[u] = e < SLOT;
        sc[u] = e / CW;
        so[u] = e % CW;
        const int o = so[u];
        int iofs, lofs;
        if (o < KB) { iofs = KB; lofs = KB - o; }
        else if (o < 2 * KB) { iofs = KB - (o - KB); lofs = KB; }
        else if (o == 2 * KB) { iofs = 1; lofs = 1 + KB; }
        else { iofs = 1 + KB; lofs = 1; }
        const int dg = k + iofs - lofs;
        inb[u] = live[u] && dg >= 0 && dg <= 2 * k;
        src[u] = band + s0 + lofs + (inb[u] ? (int64_t)dg * ld : 0);
        hi_ofs[u] = iofs > lofs ? iofs : lofs;  // beyond the partition once jj + hi_ofs >= ni
        idn[u] = iofs == lofs;
    }
    auto stage = [&](int Gs) {
        double *r = raw + (Gs % RING) * SLOT + t;
#pragma unroll
        for (int u = 0; u < NU; ++u) {
            if (!live[u]) continue;
            const int jj = Gs * TR + sc[u];
            if (inb[u] && jj + hi_ofs[u] < ni) cp_async_small<8>(r + u * NT, src[u] + jj);
            else r[u * NT] = (jj + hi_ofs[u] >= ni && idn[u]) ? 1.0 : 0.0;
        }
    };
    auto convert = [&](int Gs) {
        const double *r = raw + (Gs % RING) * SLOT + t;
        T *c = cv_ + (Gs & 1) * TR * CWP;
#pragma unroll
        for (int u = 0; u < NU; ++u) {
            if (!live[u]) continue;
            const int jj = Gs * TR + sc[u], o = so[u];
            const int pos = o < KB ? ((jj - o) & (KB - 1)) : o < 2 * KB ? KB + ((jj - (o - KB)) & (KB - 1)) : o;
            c[sc[u] * CWP + pos] = from_f64<T>(r[u * NT]);
        }
    };

    // window of columns 0..KB-1, pivot row and column 0
    T w[TR][TR];
#pragma unroll
    for (int r = 0; r < TR; ++r)
#pragma unroll
        for (int c = 0; c < TR; ++c) w[r][c] = (T)entry(ty * TR + r, tx * TR + c);
    for (int e = t; e <= 2 * KB; e += NT) {
        if (e < KB) rowb[e] = (T)entry(0, e == 0 ? KB : e);
        else if (e < 2 * KB) colb[e - KB] = (T)(e == KB ? entry(KB, 0) : entry(e - KB, 0));
        else pivb[0] = (T)entry(0, 0);
    }
    for (int e = t; e < KB * KB; e += NT)  // no L_{0,-1}
        if (e / KB <= e % KB) LT[b0 * KB * KB + e] = T(0);
    for (int Gs = 0; Gs < PD; ++Gs) {
        if (Gs < NG) stage(Gs);
        cp_async_commit();
    }
    cp_async_wait<PD - 1>();
    convert(0);
    // the three per-group tasks fall on different columns of the group
    constexpr int S_STAGE = 0, S_CONVERT = TR > 1 ? 1 : 0, S_FLUSH = TR > 2 ? 2 : 0;

    for (int Gi = 0; Gi < NG; ++Gi) {
        const int g = Gi % GRID, J = Gi / GRID;
        const bool rowg = (ty == g), colg = (tx == g);
        const T *cg = cv_ + (Gi & 1) * TR * CWP;
        T *ut_row = UT + ((b0 + J) * KB + g * TR) * KB + tx * TR;
        T *ls_blk = LS + (J & 1) * KB * LDL;
#pragma unroll
        for (int s = 0; s < TR; ++s) {
            const int j = Gi * TR + s;
            const int a = g * TR + s;  // j mod KB
            const int par = j & 1;
            __syncthreads();
            if (s == S_STAGE) {
                if (Gi + PD < NG) stage(Gi + PD);  // ring slot of group Gi-1, converted during group Gi-2
                cp_async_commit();
            }
            if (s == S_CONVERT) {
                cp_async_wait<PD - 1>();  // this thread's copies of group Gi+1 have landed
                if (Gi + 1 < NG) convert(Gi + 1);
            }
            if (s == S_FLUSH && J > 0) {  // tile rows g*TR.. of the previous block's multipliers
                const T *ls = LS + ((J - 1) & 1) * KB * LDL;
                T *lt = LT + (b0 + J - 1) * KB * KB;
                for (int e = t; e < TR * KB; e += NT) {
                    const int a2 = g * TR + e / KB, b = e % KB;
                    lt[(a2 > b ? 0 : KB * KB) + a2 * KB + b] = ls[b * LDL + a2];
                }
            }
            const T piv = pivb[par];
            T u[TR], cv[TR], nr[TR], nc[TR], m[TR];
            ld_row<T, TR>(rowb + par * KB + tx * TR, u);
            ld_row<T, TR>(colb + par * KB + ty * TR, cv);
            if (rowg) ld_row<T, TR>(cg + s * CWP + tx * TR, nr);
            if (colg) ld_row<T, TR>(cg + s * CWP + KB + ty * TR, nc);
            if (t == 0 && !usable_pivot<T>(piv))
                atomicMin((unsigned long long *)status, (unsigned long long)(s0 + j));
            const T pinv = fast_rcp<T>(piv);
#pragma unroll
            for (int r = 0; r < TR; ++r) m[r] = cv[r] * pinv;
            // row j and column j leave; row j+KB and column j+KB enter
            if (rowg) {
#pragma unroll
                for (int c = 0; c < TR; ++c) w[s][c] = nr[c];
            }
            if (colg) {
#pragma unroll
                for (int r = 0; r < TR; ++r) w[r][s] = nc[r];
            }
#pragma unroll
            for (int r = 0; r < TR; ++r)
#pragma unroll
                for (int c = 0; c < TR; ++c) w[r][c] -= m[r] * u[c];
            // outputs: multipliers (staged), scaled pivot row, 1/u_jj
            if (tx == 0) st_row<T, TR>(ls_blk + a * LDL + ty * TR, m);
            if (rowg) {
                T v[TR];
#pragma unroll
                for (int c = 0; c < TR; ++c) v[c] = u[c] * pinv;
                st_row<T, TR>(ut_row + s * KB, v);
            }
            if (t == 0) DI[b0 * KB + j] = pinv;
            // publish pivot row and column j+1
            if (j + 1 < NP) {
                const int s1 = (s + 1) % TR;
                const int g1 = (s + 1 == TR) ? (g + 1) % GRID : g;
                const int par1 = par ^ 1;
                if (ty == g1) {
                    T v[TR];
#pragma unroll
                    for (int c = 0; c < TR; ++c) v[c] = w[s1][c];
                    st_row<T, TR>(rowb + par1 * KB + tx * TR, v);
                }
                if (tx == g1) {
                    T v[TR];
#pragma unroll
                    for (int r = 0; r < TR; ++r) v[r] = w[r][s1];
                    st_row<T, TR>(colb + par1 * KB + ty * TR, v);
                }
                if (ty == g1 && tx == g1) {
                    const int a1 = g1 * TR + s1;
                    pivb[par1] = w[s1][s1];
                    rowb[par1 * KB + a1] = cg[s * CWP + 2 * KB];
                    colb[par1 * KB + a1] = cg[s * CWP + 2 * KB + 1];
                }
            }
        }
    }
    __syncthreads();
    // multipliers of the last block (no block below it)
    for (int e = t; e < KB * KB; e += NT) {
        const int a = e / KB, b = e % KB;
        if (a > b) LT[(b0 + nb - 1) * KB * KB + e] = LS[((nb - 1) & 1) * KB * LDL + b * LDL + a];
    }
}

template <typename T, int KB> struct InvGeo {
    static constexpr int H = KB / 2;                    // half size
    static constexpr int NT = 4 * H;                    // two matrices x two diagonal halves x H columns
    static constexpr int TILES = (H / 4) * (H / 4);     // 4 x 4 output tiles of one H x H product
    static constexpr int LDM = KB + 16 / (int)sizeof(T);
    static constexpr size_t bytes = (size_t)2 * KB * LDM * sizeof(T);
};

// x[0..N-1] = column c of M^{-1} for a unit lower triangular N x N matrix M
// (strictly lower part in shared memory, zero elsewhere, row stride ldm):
// x_i = [i == c] - sum_{q < i} M_iq x_q  (x_i = 0 for i < c follows).
template <typename T, int N>
__device__ __forceinline__ void tri_inv_col(const T *M, int ldm, int c, T (&x)[N]) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
        T acc0 = (i == c) ? T(1) : T(0), acc1 = T(0);
#pragma unroll
        for (int q = 0; q < i; q += 4) {
            T mv[4];
            ld_row<T, 4>(M + i * ldm + q, mv);
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (q + u < i) {
                    if (u & 1) acc1 -= mv[u] * x[q + u];
                    else acc0 -= mv[u] * x[q + u];
                }
        }
        x[i] = acc0 + acc1;
    }
}

// acc = A B over the 4 x 4 tile (i0, j0) of H x H operands (row stride ldm),
// inner index q in [q0, q1) (multiples of 4)
template <typename T>
__device__ __forceinline__ void tile4_mac(const T *A, const T *B, int ldm, int i0, int j0, int q0, int q1,
                                          T (&acc)[4][4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    for (int q = q0; q < q1; q += 4) {
        T av[4][4], bv[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i) ld_row<T, 4>(A + (i0 + i) * ldm + q, av[i]);
#pragma unroll
        for (int u = 0; u < 4; ++u) ld_row<T, 4>(B + (q + u) * ldm + j0, bv[u]);
        if constexpr (sizeof(T) == 4) {
            // two columns per packed FP32 FMA (each half rounds like fmaf)
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; j += 2) {
                        const float2 o = __ffma2_rn(make_float2(av[i][u], av[i][u]), make_float2(bv[u][j], bv[u][j + 1]),
                                                    make_float2(acc[i][j], acc[i][j + 1]));
                        acc[i][j] = o.x;
                        acc[i][j + 1] = o.y;
                    }
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] += av[i][u] * bv[u][j];
        }
    }
}

template <typename T, int KB>
__global__ void __launch_bounds__(InvGeo<T, KB>::NT) k_band_lu_inv(T *__restrict__ LT, T *__restrict__ UT) {
    using G = InvGeo<T, KB>;
    constexpr int H = G::H, NT = G::NT, LDM = G::LDM, TILES = G::TILES;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *Ms = reinterpret_cast<T *>(smem_raw);  // [2][KB][LDM]: L_JJ, P (D^{-1}U_JJ) P; inverted in place
    T *lt = LT + (int64_t)blockIdx.x * KB * KB, *ut = UT + (int64_t)blockIdx.x * KB * KB;
    const int t = threadIdx.x;
    // 4-vectors of a tile row: (a, b..b+3); U is stored reversed, so its
    // vector lands at columns KB-4-b.. in reverse order
    constexpr int C4 = KB * KB / 4;
    for (int e = t; e < C4; e += NT) {
        const int a = (4 * e) / KB, b = (4 * e) % KB;
        T lv[4], uv[4], lo[4], uo[4];
        ld_row<T, 4>(lt + 4 * e, lv);
        ld_row<T, 4>(ut + 4 * e, uv);
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            lo[w] = (a > b + w) ? lv[w] : T(0);
            uo[3 - w] = (a < b + w) ? uv[w] : T(0);
        }
        st_row<T, 4>(Ms + a * LDM + b, lo);
        st_row<T, 4>(Ms + KB * LDM + (KB - 1 - a) * LDM + (KB - 4 - b), uo);
    }
    __syncthreads();
    // diagonal halves: thread t -> matrix t / 2H, half (t / H) % 2, column t % H
    {
        const int c = t % H;
        T *Md = Ms + (t / (2 * H)) * KB * LDM + ((t / H) % 2) * H * (LDM + 1);
        T x[H];
        tri_inv_col<T, H>(Md, LDM, c, x);
        __syncthreads();
#pragma unroll
        for (int i = 0; i < H; ++i)
            if (i >= c) Md[i * LDM + c] = (i == c) ? T(1) : x[i];  // unit diagonal kept for the products
        __syncthreads();
    }
    // off-diagonal half: T21 = M21 X11 (X11 lower: q >= j0), then X21 = -X22 T21 (X22 lower: q <= i0 + 3).
    // The trip count of the first product depends on the tile column, of the second on
    // the tile row: tiles go column-major, then row-major, so that a warp's tiles agree.
    const bool act = t < 2 * TILES;
    T *Mm = Ms + (t / TILES) * KB * LDM;
    const int tile = t % TILES, ta = tile / (H / 4), tb = tile % (H / 4);
    T *X11 = Mm, *M21 = Mm + H * LDM, *X22 = Mm + H * LDM + H;
    T acc[4][4];
    {
        // KB = 64 (8 x 8 tiles per product): the same 32 tiles per warp, lanes
        // reassigned so that a quarter-warp takes four tile columns of two tile
        // rows, whose M21 rows (4 apart) fall on disjoint bank halves (the map
        // above puts eight rows on two bank groups); smaller blocks keep it
        const int tp = (H == 32) ? ((tile & ~31) | ((tile & 3) << 3) | ((tile >> 2) & 7)) : tile;
        const int pa = tp / (H / 4), pb = tp % (H / 4);
        if (act) tile4_mac<T>(M21, X11, LDM, pb * 4, pa * 4, pa * 4, H, acc);
        __syncthreads();
        if (act) {
#pragma unroll
            for (int i = 0; i < 4; ++i) st_row<T, 4>(M21 + (pb * 4 + i) * LDM + pa * 4, acc[i]);
        }
    }
    __syncthreads();
    const int i0 = ta * 4, j0 = tb * 4;
    if (act) tile4_mac<T>(X22, M21, LDM, i0, j0, 0, i0 + 4, acc);
    __syncthreads();
    if (act) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            T v[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) v[j] = -acc[i][j];
            st_row<T, 4>(M21 + (i0 + i) * LDM + j0, v);
        }
    }
    __syncthreads();
    // strict triangles back: whole 4-vectors inside a triangle, single entries on its edge
    for (int e = t; e < C4; e += NT) {
        const int a = (4 * e) / KB, b = (4 * e) % KB;
        T lv[4], uv[4], ur_[4];
        ld_row<T, 4>(Ms + a * LDM + b, lv);
        ld_row<T, 4>(Ms + KB * LDM + (KB - 1 - a) * LDM + (KB - 4 - b), ur_);
#pragma unroll
        for (int w = 0; w < 4; ++w) uv[w] = ur_[3 - w];
        if (b + 3 < a) st_row<T, 4>(lt + 4 * e, lv);
        else if (b > a) st_row<T, 4>(ut + 4 * e, uv);
        else {
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                if (a > b + w) lt[4 * e + w] = lv[w];
                else if (a < b + w) ut[4 * e + w] = uv[w];
            }
        }
    }
}

template <typename T, int KB>
static bool col_impl(Ctx *c) {
    // partitions [g0, g1): a Parts view starting at g0 (the kernels index
    // rows and blocks through the offsets, which stay global)
    const int g0 = c->lu_g1 < 0 ? 0 : c->lu_g0, g1 = c->lu_g1 < 0 ? c->p : c->lu_g1;
    const int64_t b0 = c->boff_h[g0], nb = c->boff_h[g1] - b0;
    Parts P{c->off_d + g0, c->boff_d + g0, g1 - g0};
    const size_t sm1 = ColSmem<T, KB>::bytes, sm2 = InvGeo<T, KB>::bytes;
    if constexpr (sizeof(T) == 4)
        cudaFuncSetAttribute(k_band_lu_col<T, KB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
    cudaFuncSetAttribute(k_band_lu_inv<T, KB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
    if constexpr (sizeof(T) == 8) {
        const size_t smc = Col1Smem<T, KB>::bytes;
        cudaFuncSetAttribute(k_band_lu_col1<T, KB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smc);
        if (!launch(c, KID_LU, [&] {
                k_band_lu_col1<T, KB><<<g1 - g0, Col1Geo<T, KB>::NT, smc, c->stream>>>(
                    c->band, c->ld, c->k, P, (T *)c->LT, (T *)c->UT, (T *)c->DI, c->status);
            }))
            return false;
    } else if (!launch(c, KID_LU, [&] {
                   k_band_lu_col<T, KB><<<g1 - g0, ColGeo<T, KB>::NT, sm1, c->stream>>>(
                       c->band, c->ld, c->k, P, (T *)c->LT, (T *)c->UT, (T *)c->DI, c->status);
               }))
        return false;
    return launch(c, KID_LU_INV, [&] {
        k_band_lu_inv<T, KB><<<(unsigned)nb, InvGeo<T, KB>::NT, sm2, c->stream>>>(
            (T *)c->LT + b0 * KB * KB, (T *)c->UT + b0 * KB * KB);
    });
}

template <typename T>
static bool col_kb(Ctx *c) {
    switch (c->KB) {
        case 8: return col_impl<T, 8>(c);
        case 16: return col_impl<T, 16>(c);
        case 32: return col_impl<T, 32>(c);
        default: return col_impl<T, 64>(c);
    }
}

bool run_band_lu_col(Ctx *c) { return c->fp64 ? col_kb<double>(c) : col_kb<float>(c); }

}  // namespace lrs
