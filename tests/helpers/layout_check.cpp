// Host check of the column pass's per-warp scratch layout (make_layout in
// colpass_shape.cuh): for every pass kind, value size, cap 1..80, A row
// width 1..40, with and without diagonal slots and the Pi buffers, every
// buffer lies inside the warp's bytes at a 16-byte boundary, and no two
// buffers overlap unless their lifetimes are disjoint by design:
//   tie rows / union table   (a drop runs after its union)
//   R list / union, S, T      (the update phase ends before R is formed;
//                              T only with A in diagonal slots)
//   LOMR table B / union, tie, histogram (table B is empty until A P)
//   CG pass B's table A / union, tie, histogram; union / histogram (A's keys
//                              are cleared before A P; the union is over
//                              before the selection)
// Prints the number of violations; exit status 1 if there is any.
#include <cstdio>
#include <string>
#include <vector>

#include "colpass_shape.cuh"

using namespace spai;

struct Buf {
  std::string name;
  int lo, hi;
};

int main() {
  long bad = 0, cases = 0;
  for (int kind = 0; kind <= 5; kind++)
    for (int vc : {4, 8})
      for (int CAP = 1; CAP <= 80; CAP++)
        for (int W = 1; W <= 40; W++)
          for (int dia = 0; dia <= 1; dia++)
            for (int pi = 0; pi <= 1; pi++) {
              WarpLayout L = make_layout(kind, vc, CAP, W, dia != 0, pi != 0);
              const int LMAX = CAP * W + 1;
              int TMAX = 2 * CAP;
              if (kind == kLOMR) TMAX = 3 * CAP;
              if (kind == kCGB) TMAX = LMAX + CAP;
              const int LIST = LMAX > TMAX ? LMAX : TMAX;
              const bool lomr = kind == kLOMR, hasP = kind != kRES;
              const bool upd = kind == kMR || kind == kLOMR || kind == kCGA;
              std::vector<Buf> b = {{"R", L.Rr, L.Rv + vc * LMAX},
                                    {"A", L.hk, L.ho + 2 * L.H},
                                    {"M", L.Mr, L.Mv + vc * CAP},
                                    {"T", L.Tr, L.Tv + vc * TMAX},
                                    {"U", L.uk, L.uo + 2 * L.HU},
                                    {"tie", L.tie, L.tie + 4 * LIST},
                                    {"hist", L.hist, L.hist + 512}};
              if (hasP) b.push_back({"P", L.Pr, L.Pv + vc * CAP});
              if (lomr) {
                b.push_back({"B", L.gk, L.go + 2 * L.H});
                b.push_back({"Z", L.Zr, L.Zv + vc * CAP});
                b.push_back({"S", L.Sr, L.Sv + vc * 2 * CAP});
              }
              if (pi) b.push_back({"pi", L.zr, L.zv + vc * LMAX});
              auto allowed = [&](const std::string& x, const std::string& y) {
                auto is = [&](const char* p, const char* q) {
                  return (x == p && y == q) || (x == q && y == p);
                };
                if (is("tie", "U")) return true;
                if (upd && (is("R", "U") || is("R", "S"))) return true;
                if (upd && dia && is("R", "T")) return true;
                if (lomr && (is("B", "U") || is("B", "tie") || is("B", "hist"))) return true;
                if (kind == kCGB && (is("A", "U") || is("A", "tie") || is("A", "hist") ||
                                     is("U", "hist")))
                  return true;
                return false;
              };
              cases++;
              for (auto& x : b)
                if (x.lo < 0 || x.hi > L.bytes || x.lo % 16) {
                  if (bad++ < 10)
                    printf("outside: %s kind %d vc %d cap %d W %d dia %d\n", x.name.c_str(), kind,
                           vc, CAP, W, dia);
                }
              for (size_t i = 0; i < b.size(); i++)
                for (size_t j = i + 1; j < b.size(); j++)
                  if (b[i].lo < b[j].hi && b[j].lo < b[i].hi && !allowed(b[i].name, b[j].name)) {
                    if (bad++ < 10)
                      printf("overlap: %s %s kind %d vc %d cap %d W %d dia %d pi %d\n",
                             b[i].name.c_str(), b[j].name.c_str(), kind, vc, CAP, W, dia, pi);
                  }
            }
  printf("cases %ld violations %ld\n", cases, bad);
  return bad != 0;
}
