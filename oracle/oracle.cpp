// TrioSeq oracle — TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, obviously-correct CPU implementation of exact 3-way alignment under
// sum-of-pairs scoring with a linear gap, written from the paper's definitions:
//   * the recurrence, Eq. 1 (Sec. II): each cell M[i][j][k] is the best of its 7 predecessors
//     plus the sum-of-pairs (SOP) score of the column that the move emits;
//   * the SOP of a column, Sec. II: sigma(x,y) + sigma(x,z) + sigma(y,z) with sigma(residue, gap)
//     = alpha and sigma(gap, gap) = 0;
//   * global alignment, Sec. II "Global Alignments": M[0][0][0] = 0, v = -infinity (realised here
//     by skipping predecessors outside the cube, which reproduces the face recurrences and the
//     axis values 2*i*alpha), score = M[a][b][c];
//   * semi-global and local alignment, Sec. II "Semi-Global Alignments" / "Local Alignments"
//     (score only, oracle_align_type).
// Tie-break (the paper is silent): the first maximal candidate in Eq. 1's listing order wins,
// i.e. (1,1,1) > (1,1,0) > (1,0,1) > (0,1,1) > (1,0,0) > (0,1,0) > (0,0,1).
//
// Only tests/, the package smoke check and the benchmark's CPU-baseline leg may load this
// library; the product path never does. It shares no code with the CUDA path.
//
// Arithmetic is int64 throughout, so it cannot overflow for any input the library accepts.
// Residues are codes 0..K-1; in emitted alignment rows, the gap is ORACLE_GAP (255).

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>

namespace {

constexpr uint8_t ORACLE_GAP = 255;

// Moves in Eq. 1's listing order: (di, dj, dk).
constexpr int kMoves[7][3] = {
    {1, 1, 1}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};

struct Scoring {
  int K;
  const int32_t* sub;  // K*K row-major, symmetric
  int64_t gap;         // alpha
  // sigma over residues and gaps (Sec. II): residue/residue from the matrix, residue/gap = alpha,
  // gap/gap = 0.
  int64_t sigma(int x, int y) const {
    if (x < 0 && y < 0) return 0;
    if (x < 0 || y < 0) return gap;
    return sub[x * K + y];
  }
  // SOP of one column (x, y, z); -1 stands for a gap.
  int64_t sop(int x, int y, int z) const { return sigma(x, y) + sigma(x, z) + sigma(y, z); }
};

}  // namespace

extern "C" {

// Exact 3-way global alignment (Eq. 1, global initialisation of Sec. II).
//   s0/s1/s2: residue codes, lengths a/b/c (any may be 0).
//   K, sub: alphabet size and K*K symmetric substitution matrix; gap: alpha (<= 0 in practice).
//   score_out: M[a][b][c].
//   If rows != nullptr, the optimal alignment under the tie-break above is written to
//   rows[0..L), rows[cap..cap+L), rows[2cap..2cap+L) (gap = 255) and L to *len_out;
//   requires cap >= a+b+c. Returns 0 on success, -1 on bad arguments, -2 on allocation failure.
int oracle_align(const uint8_t* s0, int a, const uint8_t* s1, int b, const uint8_t* s2, int c,
                 int K, const int32_t* sub, int32_t gap, int64_t* score_out, uint8_t* rows,
                 int64_t cap, int64_t* len_out) {
  if (a < 0 || b < 0 || c < 0 || K <= 0 || !sub || !score_out) return -1;
  if (rows && cap < (int64_t)a + b + c) return -1;
  Scoring sc{K, sub, gap};
  const int64_t B = b + 1, C = c + 1;
  const int64_t plane = B * C;
  const bool want_tb = rows != nullptr;
  std::vector<uint8_t> code;  // full cube of winning-move indices (0..6), 7 = origin
  try {
    if (want_tb) code.assign((size_t)(a + 1) * (size_t)plane, 7);
  } catch (...) {
    return -2;
  }
  // Two i-slices of scores suffice for the values (each move goes back at most one slice in i).
  std::vector<int64_t> prev(plane), cur(plane);
  for (int i = 0; i <= a; i++) {
    for (int j = 0; j <= b; j++) {
      for (int k = 0; k <= c; k++) {
        int64_t best = 0;
        int arg = 7;
        if (i == 0 && j == 0 && k == 0) {
          best = 0;  // M_000 = 0
        } else {
          bool have = false;
          for (int m = 0; m < 7; m++) {
            const int di = kMoves[m][0], dj = kMoves[m][1], dk = kMoves[m][2];
            const int pi = i - di, pj = j - dj, pk = k - dk;
            if (pi < 0 || pj < 0 || pk < 0) continue;  // v = -infinity: predecessor outside cube
            const int64_t pv = (di ? prev : cur)[(int64_t)pj * C + pk];
            const int x = di ? (int)s0[i - 1] : -1;
            const int y = dj ? (int)s1[j - 1] : -1;
            const int z = dk ? (int)s2[k - 1] : -1;
            const int64_t cand = pv + sc.sop(x, y, z);
            if (!have || cand > best) {  // strict '>' keeps the first maximal move
              best = cand;
              arg = m;
              have = true;
            }
          }
        }
        cur[(int64_t)j * C + k] = best;
        if (want_tb) code[(size_t)i * plane + (size_t)j * C + k] = (uint8_t)arg;
      }
    }
    std::swap(prev, cur);
  }
  *score_out = prev[(int64_t)b * C + c];
  if (!want_tb) return 0;
  // Traceback: from (a,b,c) follow the stored winning moves to the origin, emitting columns in
  // reverse, then reverse them.
  std::vector<uint8_t> r0, r1, r2;
  int i = a, j = b, k = c;
  while (i > 0 || j > 0 || k > 0) {
    const int m = code[(size_t)i * plane + (size_t)j * C + k];
    if (m > 6) return -1;  // cannot happen for a well-formed cube
    const int di = kMoves[m][0], dj = kMoves[m][1], dk = kMoves[m][2];
    r0.push_back(di ? s0[i - 1] : ORACLE_GAP);
    r1.push_back(dj ? s1[j - 1] : ORACLE_GAP);
    r2.push_back(dk ? s2[k - 1] : ORACLE_GAP);
    i -= di; j -= dj; k -= dk;
  }
  const int64_t L = (int64_t)r0.size();
  for (int64_t t = 0; t < L; t++) {
    rows[t] = r0[L - 1 - t];
    rows[cap + t] = r1[L - 1 - t];
    rows[2 * cap + t] = r2[L - 1 - t];
  }
  *len_out = L;
  return 0;
}

// Score of the three alignment types of Sec. II (score only).
//   type 0, "Global Alignments": as oracle_align.
//   type 1, "Semi-Global Alignments": the axes are initialised to zero,
//     M[i][0][0] = M[0][j][0] = M[0][0][k] = 0 (the origin included); every other cell follows
//     Eq. 1 with v = -infinity; the score is the best cell on a last slice in any direction,
//     max of M over the cells with i = a or j = b or k = c.
//   type 2, "Local Alignments": the same zero axes, and v = 0 in Eq. 1 for every other cell
//     (no cell is negative); the score is the best cell of the whole cube.
// Returns 0, or -1 on bad arguments.
int oracle_align_type(const uint8_t* s0, int a, const uint8_t* s1, int b, const uint8_t* s2,
                      int c, int K, const int32_t* sub, int32_t gap, int type,
                      int64_t* score_out) {
  if (a < 0 || b < 0 || c < 0 || K <= 0 || !sub || !score_out || type < 0 || type > 2) return -1;
  if (type == 0)
    return oracle_align(s0, a, s1, b, s2, c, K, sub, gap, score_out, nullptr, 0, nullptr);
  Scoring sc{K, sub, gap};
  const int64_t C = c + 1;
  const int64_t plane = (int64_t)(b + 1) * C;
  std::vector<int64_t> prev(plane), cur(plane);
  bool have_score = false;
  int64_t score = 0;
  for (int i = 0; i <= a; i++) {
    for (int j = 0; j <= b; j++) {
      for (int k = 0; k <= c; k++) {
        const int zeros = (i == 0) + (j == 0) + (k == 0);
        int64_t best = 0;
        if (zeros >= 2) {
          best = 0;  // zero-initialised axes (and origin)
        } else {
          bool have = false;
          for (int m = 0; m < 7; m++) {
            const int di = kMoves[m][0], dj = kMoves[m][1], dk = kMoves[m][2];
            const int pi = i - di, pj = j - dj, pk = k - dk;
            if (pi < 0 || pj < 0 || pk < 0) continue;
            const int64_t pv = (di ? prev : cur)[(int64_t)pj * C + pk];
            const int x = di ? (int)s0[i - 1] : -1;
            const int y = dj ? (int)s1[j - 1] : -1;
            const int z = dk ? (int)s2[k - 1] : -1;
            const int64_t cand = pv + sc.sop(x, y, z);
            if (!have || cand > best) {
              best = cand;
              have = true;
            }
          }
          if (type == 2 && best < 0) best = 0;  // v = 0
        }
        cur[(int64_t)j * C + k] = best;
        const bool counts = type == 2 || i == a || j == b || k == c;
        if (counts && (!have_score || best > score)) {
          score = best;
          have_score = true;
        }
      }
    }
    std::swap(prev, cur);
  }
  *score_out = score;
  return 0;
}

// Score and alignment of the three alignment types of Sec. II, with the span of the cube the
// alignment covers: begin[3] = (i0, j0, k0), end[3] = (i1, j1, k1); the rows align
// S0[i0:i1], S1[j0:j1], S2[k0:k1] (columns of the path from begin to end).
//   type 0 (global): as oracle_align; begin = (0,0,0), end = (a,b,c).
//   type 1 (semi-global) and 2 (local): the cube as in oracle_align_type. The end cell is the
//     first cell in (i, j, k) order holding the best score among the cells that count (the last
//     faces for semi-global, every cell for local). From it the walk follows, at each cell, the
//     first maximal candidate in Eq. 1's listing order, v being listed last: the walk stops at an
//     axis cell (two zero indices, initialised, not computed) and, for local, where v = 0 is the
//     only maximal candidate.
// rows/cap/len_out as in oracle_align (cap >= a+b+c). Returns 0, -1 (bad arguments), -2.
int oracle_align_type_tb(const uint8_t* s0, int a, const uint8_t* s1, int b, const uint8_t* s2,
                         int c, int K, const int32_t* sub, int32_t gap, int type,
                         int64_t* score_out, uint8_t* rows, int64_t cap, int64_t* len_out,
                         int32_t* begin, int32_t* end) {
  if (a < 0 || b < 0 || c < 0 || K <= 0 || !sub || !score_out || !rows || !len_out || !begin ||
      !end || type < 0 || type > 2 || cap < (int64_t)a + b + c)
    return -1;
  if (type == 0) {
    const int rc = oracle_align(s0, a, s1, b, s2, c, K, sub, gap, score_out, rows, cap, len_out);
    begin[0] = begin[1] = begin[2] = 0;
    end[0] = a;
    end[1] = b;
    end[2] = c;
    return rc;
  }
  Scoring sc{K, sub, gap};
  const int64_t C = c + 1, plane = (int64_t)(b + 1) * C;
  std::vector<uint8_t> code;  // winning move 0..6, or 7 = start here (axis cell, or v won)
  try {
    code.assign((size_t)(a + 1) * (size_t)plane, 7);
  } catch (...) {
    return -2;
  }
  std::vector<int64_t> prev(plane), cur(plane);
  bool have_score = false;
  int64_t score = 0;
  int ei = 0, ej = 0, ek = 0;
  for (int i = 0; i <= a; i++) {
    for (int j = 0; j <= b; j++) {
      for (int k = 0; k <= c; k++) {
        const int zeros = (i == 0) + (j == 0) + (k == 0);
        int64_t best = 0;
        int arg = 7;
        if (zeros < 2) {
          bool have = false;
          for (int m = 0; m < 7; m++) {
            const int di = kMoves[m][0], dj = kMoves[m][1], dk = kMoves[m][2];
            const int pi = i - di, pj = j - dj, pk = k - dk;
            if (pi < 0 || pj < 0 || pk < 0) continue;
            const int64_t pv = (di ? prev : cur)[(int64_t)pj * C + pk];
            const int x = di ? (int)s0[i - 1] : -1;
            const int y = dj ? (int)s1[j - 1] : -1;
            const int z = dk ? (int)s2[k - 1] : -1;
            const int64_t cand = pv + sc.sop(x, y, z);
            if (!have || cand > best) {
              best = cand;
              arg = m;
              have = true;
            }
          }
          if (type == 2 && best < 0) {  // v = 0 is listed last: it wins only when alone
            best = 0;
            arg = 7;
          }
        }
        cur[(int64_t)j * C + k] = best;
        code[(size_t)i * plane + (size_t)j * C + k] = (uint8_t)arg;
        const bool counts = type == 2 || i == a || j == b || k == c;
        if (counts && (!have_score || best > score)) {  // first cell with the best score
          score = best;
          have_score = true;
          ei = i;
          ej = j;
          ek = k;
        }
      }
    }
    std::swap(prev, cur);
  }
  *score_out = score;
  std::vector<uint8_t> r0, r1, r2;
  int i = ei, j = ej, k = ek;
  for (;;) {
    const int m = code[(size_t)i * plane + (size_t)j * C + k];
    if (m > 6) break;  // start cell
    const int di = kMoves[m][0], dj = kMoves[m][1], dk = kMoves[m][2];
    r0.push_back(di ? s0[i - 1] : ORACLE_GAP);
    r1.push_back(dj ? s1[j - 1] : ORACLE_GAP);
    r2.push_back(dk ? s2[k - 1] : ORACLE_GAP);
    i -= di;
    j -= dj;
    k -= dk;
  }
  const int64_t L = (int64_t)r0.size();
  for (int64_t t = 0; t < L; t++) {
    rows[t] = r0[L - 1 - t];
    rows[cap + t] = r1[L - 1 - t];
    rows[2 * cap + t] = r2[L - 1 - t];
  }
  *len_out = L;
  begin[0] = i;
  begin[1] = j;
  begin[2] = k;
  end[0] = ei;
  end[1] = ej;
  end[2] = ek;
  return 0;
}

// ---------------------------------------------------------------------------------------------
// Affine gaps (the paper's future work, Sec. VI; no definition is given there). Reading: the
// sum-of-pairs score with natural gap costs (Altschul 1989) in Gotoh's affine form (Gotoh 1982,
// 1986): the score of a 3-way alignment is the sum, over the three pairs (p, q), of the score of
// the pairwise alignment it induces on (p, q) once the columns with a gap in both p and q are
// deleted. That pairwise score is sigma(x, y) per residue pair, alpha per residue aligned to a gap
// (the linear term of Sec. II), and gamma (gap_open, <= 0) once per maximal run of consecutive
// induced columns with a gap in the same sequence. With gamma = 0 it is Eq. 1's score.
//
// Dynamic program. The state of an alignment prefix records, for each pair, the kind of its last
// induced column: 0 = both residues (or no column yet), 1 = gap in the pair's first sequence,
// 2 = gap in its second. A new column of move m leaves a pair's state unchanged where m has a gap
// in both sequences of the pair, and otherwise sets it; it opens a run (gamma) where it has a gap
// in one sequence of the pair and the pair's state is not already a gap in that sequence.
// F[i][j][k][s] = best score of the prefixes ending in state s; F[0][0][0][all zero] = 0.
namespace {

constexpr int kPairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};
constexpr int64_t kNoState = INT64_MIN / 4;  // F of a state no prefix ends in

inline int state_index(const int st[3]) { return st[0] * 9 + st[1] * 3 + st[2]; }

// Column m (residues x, y, z or -1 for a gap) appended to state `from`: its score and new state.
int64_t affine_step(const Scoring& sc, int64_t gamma, int from, const int v[3], int* to) {
  int st[3] = {from / 9, (from / 3) % 3, from % 3};
  int64_t cost = 0;
  for (int q = 0; q < 3; q++) {
    const int p0 = kPairs[q][0], p1 = kPairs[q][1];
    const bool r0 = v[p0] >= 0, r1 = v[p1] >= 0;
    if (!r0 && !r1) continue;  // deleted from this pair's induced alignment
    if (r0 && r1) {
      cost += sc.sub[v[p0] * sc.K + v[p1]];
      st[q] = 0;
    } else {
      const int kind = r0 ? 2 : 1;  // 1: gap in p0, 2: gap in p1
      cost += sc.gap + (st[q] == kind ? 0 : gamma);
      st[q] = kind;
    }
  }
  *to = state_index(st);
  return cost;
}

}  // namespace

// Exact 3-way global alignment score under affine gaps with natural gap costs (above).
//   gap: alpha (per residue aligned to a gap), gap_open: gamma (per maximal gap run of a pair).
//   If rows != nullptr the alignment is emitted as in oracle_align (cap >= a+b+c); the end state
//   is the first maximal state in index order, and the walk back takes, at each (cell, state), the
//   first maximal (move in Eq. 1's listing order, previous state in index order).
// Returns 0, -1 (bad arguments) or -2 (allocation failure).
int oracle_align_affine(const uint8_t* s0, int a, const uint8_t* s1, int b, const uint8_t* s2,
                        int c, int K, const int32_t* sub, int32_t gap, int32_t gap_open,
                        int64_t* score_out, uint8_t* rows, int64_t cap, int64_t* len_out) {
  if (a < 0 || b < 0 || c < 0 || K <= 0 || !sub || !score_out) return -1;
  if (rows && (cap < (int64_t)a + b + c || !len_out)) return -1;
  Scoring sc{K, sub, gap};
  const int64_t C = c + 1, plane = (int64_t)(b + 1) * C;
  const bool want_tb = rows != nullptr;
  // traceback: per (cell, state) the winning (move * 27 + previous state), 255 = none
  std::vector<uint16_t> from;
  try {
    if (want_tb) from.assign((size_t)(a + 1) * (size_t)plane * 27, 0xFFFF);
  } catch (...) {
    return -2;
  }
  std::vector<int64_t> prev(plane * 27, kNoState), cur(plane * 27, kNoState);
  for (int i = 0; i <= a; i++) {
    for (int j = 0; j <= b; j++) {
      for (int k = 0; k <= c; k++) {
        int64_t* F = &cur[((int64_t)j * C + k) * 27];
        for (int s = 0; s < 27; s++) F[s] = kNoState;
        if (i == 0 && j == 0 && k == 0) {
          F[0] = 0;
          continue;
        }
        for (int m = 0; m < 7; m++) {
          const int di = kMoves[m][0], dj = kMoves[m][1], dk = kMoves[m][2];
          if (i - di < 0 || j - dj < 0 || k - dk < 0) continue;
          const int64_t* G = &(di ? prev : cur)[((int64_t)(j - dj) * C + (k - dk)) * 27];
          const int v[3] = {di ? (int)s0[i - 1] : -1, dj ? (int)s1[j - 1] : -1,
                            dk ? (int)s2[k - 1] : -1};
          for (int s = 0; s < 27; s++) {
            if (G[s] == kNoState) continue;
            int to = 0;
            const int64_t cand = G[s] + affine_step(sc, gap_open, s, v, &to);
            if (cand > F[to]) {  // strict: the first maximal (move, state) is kept
              F[to] = cand;
              if (want_tb)
                from[((size_t)i * plane + (size_t)j * C + k) * 27 + to] = (uint16_t)(m * 27 + s);
            }
          }
        }
      }
    }
    std::swap(prev, cur);
  }
  const int64_t* E = &prev[((int64_t)b * C + c) * 27];
  int best_s = 0;
  for (int s = 1; s < 27; s++)
    if (E[s] > E[best_s]) best_s = s;
  *score_out = E[best_s];
  if (!want_tb) return 0;
  std::vector<uint8_t> r0, r1, r2;
  int i = a, j = b, k = c, s = best_s;
  while (i > 0 || j > 0 || k > 0) {
    const uint16_t f = from[((size_t)i * plane + (size_t)j * C + k) * 27 + s];
    if (f == 0xFFFF) return -1;  // cannot happen for a reachable state
    const int m = f / 27, ps = f % 27;
    const int di = kMoves[m][0], dj = kMoves[m][1], dk = kMoves[m][2];
    r0.push_back(di ? s0[i - 1] : ORACLE_GAP);
    r1.push_back(dj ? s1[j - 1] : ORACLE_GAP);
    r2.push_back(dk ? s2[k - 1] : ORACLE_GAP);
    i -= di;
    j -= dj;
    k -= dk;
    s = ps;
  }
  const int64_t L = (int64_t)r0.size();
  for (int64_t t = 0; t < L; t++) {
    rows[t] = r0[L - 1 - t];
    rows[cap + t] = r1[L - 1 - t];
    rows[2 * cap + t] = r2[L - 1 - t];
  }
  *len_out = L;
  return 0;
}

// Textbook pairwise alignment with affine gaps (Gotoh 1982): three matrices (ending in a residue
// pair, in a gap in x, in a gap in y); a gap run of length l scores gap_open + l * gap. Used by the
// affine oracle's pins (one-empty reduction, pairwise upper bound).
int oracle_gotoh2(const uint8_t* x, int a, const uint8_t* y, int b, int K, const int32_t* sub,
                  int32_t gap, int32_t gap_open, int64_t* score_out) {
  if (a < 0 || b < 0 || !score_out) return -1;
  const int64_t NEG = INT64_MIN / 4;
  std::vector<int64_t> Mp(b + 1, NEG), Xp(b + 1, NEG), Yp(b + 1, NEG);
  std::vector<int64_t> Mc(b + 1), Xc(b + 1), Yc(b + 1);
  // row 0: M = 0 at (0,0); a gap in x (y consumed) along j
  Mp[0] = 0;
  for (int j = 1; j <= b; j++) Xp[j] = (int64_t)gap_open + (int64_t)j * gap;
  for (int i = 1; i <= a; i++) {
    Mc[0] = NEG;
    Xc[0] = NEG;
    Yc[0] = (int64_t)gap_open + (int64_t)i * gap;  // gap in y (x consumed)
    for (int j = 1; j <= b; j++) {
      const int64_t best_prev = std::max(Mp[j - 1], std::max(Xp[j - 1], Yp[j - 1]));
      Mc[j] = best_prev + sub[x[i - 1] * K + y[j - 1]];
      // gap in x: y[j-1] against a gap; extends a gap in x or opens one
      Xc[j] = std::max(Xc[j - 1] + gap, std::max(Mc[j - 1], Yc[j - 1]) + gap_open + gap);
      // gap in y: x[i-1] against a gap
      Yc[j] = std::max(Yp[j] + gap, std::max(Mp[j], Xp[j]) + gap_open + gap);
    }
    std::swap(Mp, Mc);
    std::swap(Xp, Xc);
    std::swap(Yp, Yc);
  }
  *score_out = std::max(Mp[b], std::max(Xp[b], Yp[b]));
  return 0;
}

// Sum-of-pairs score of a given 3-row alignment (Sec. II SOP summed over columns).
// rows: 3 rows of length L at stride cap, gap = 255. Returns 0, or -1 on a residue >= K.
int oracle_sp_score(const uint8_t* rows, int64_t L, int64_t cap, int K, const int32_t* sub,
                    int32_t gap, int64_t* score_out) {
  Scoring sc{K, sub, gap};
  int64_t s = 0;
  for (int64_t t = 0; t < L; t++) {
    int v[3];
    for (int q = 0; q < 3; q++) {
      const uint8_t r = rows[q * cap + t];
      if (r == ORACLE_GAP) v[q] = -1;
      else if (r < K) v[q] = r;
      else return -1;
    }
    s += sc.sop(v[0], v[1], v[2]);
  }
  *score_out = s;
  return 0;
}

// Textbook pairwise Needleman-Wunsch with a linear gap: one alpha per residue aligned to a gap.
// Used by the oracle's pins (one-empty reduction, pairwise upper bound).
int oracle_nw2(const uint8_t* x, int a, const uint8_t* y, int b, int K, const int32_t* sub,
               int32_t gap, int64_t* score_out) {
  if (a < 0 || b < 0) return -1;
  std::vector<int64_t> prev(b + 1), cur(b + 1);
  for (int j = 0; j <= b; j++) prev[j] = (int64_t)j * gap;
  for (int i = 1; i <= a; i++) {
    cur[0] = (int64_t)i * gap;
    for (int j = 1; j <= b; j++) {
      const int64_t d = prev[j - 1] + sub[x[i - 1] * K + y[j - 1]];
      const int64_t u = prev[j] + gap;
      const int64_t l = cur[j - 1] + gap;
      cur[j] = std::max(d, std::max(u, l));
    }
    std::swap(prev, cur);
  }
  *score_out = prev[b];
  return 0;
}

// Batch convenience: scores of n triplets (score only), sequences packed back to back.
// offs[3*t+q] / lens[3*t+q] locate sequence q of triplet t in `codes`.
int oracle_align_many(const uint8_t* codes, const int64_t* offs, const int32_t* lens, int64_t n,
                      int K, const int32_t* sub, int32_t gap, int64_t* scores) {
  for (int64_t t = 0; t < n; t++) {
    const int rc = oracle_align(codes + offs[3 * t], lens[3 * t], codes + offs[3 * t + 1],
                                lens[3 * t + 1], codes + offs[3 * t + 2], lens[3 * t + 2], K, sub,
                                gap, &scores[t], nullptr, 0, nullptr);
    if (rc) return rc;
  }
  return 0;
}

// The same on `nthreads` host threads: independent triplets, taken one at a time from a shared
// counter (the plain per-triplet DP above, run concurrently). Used for the all-core CPU baseline.
int oracle_align_many_mt(const uint8_t* codes, const int64_t* offs, const int32_t* lens, int64_t n,
                         int K, const int32_t* sub, int32_t gap, int64_t* scores, int nthreads) {
  std::atomic<int64_t> next{0};
  std::atomic<int> rc{0};
  const auto work = [&]() {
    for (int64_t t = next++; t < n; t = next++) {
      const int r = oracle_align(codes + offs[3 * t], lens[3 * t], codes + offs[3 * t + 1],
                                 lens[3 * t + 1], codes + offs[3 * t + 2], lens[3 * t + 2], K,
                                 sub, gap, &scores[t], nullptr, 0, nullptr);
      if (r) rc = r;
    }
  };
  std::vector<std::thread> pool;
  for (int i = 1; i < std::max(1, nthreads); i++) pool.emplace_back(work);
  work();
  for (auto& th : pool) th.join();
  return rc;
}

}  // extern "C"
