// Test harness (host only): the library's reference-element tables (csrc/refelem.cpp) for one
// (dim, space, order, basis), written in binary for the CPU tests.
// Output: int32 rc, and for rc == 0: int32 nloc, ncomp, nq, then double R[9 * nloc * nloc]
// (blocks (a, b) of int_ref phi^a phi^b, a, b < 3) and double Bdiv[nq * nloc].
#include <cstdio>
#include <cstdlib>

#include "refelem.h"

int main(int argc, char** argv) {
    if (argc != 6) return 2;
    bras::RefTables t;
    const int rc = bras::build_reference(atoi(argv[1]), atoi(argv[2]), atoi(argv[3]), &t, atoi(argv[4]));
    FILE* out = fopen(argv[5], "wb");
    if (!out) return 2;
    fwrite(&rc, sizeof(int), 1, out);
    if (rc == 0) {
        const int hdr[3] = {t.nloc, t.ncomp, t.nq};
        fwrite(hdr, sizeof(int), 3, out);
        fwrite(t.R.data(), sizeof(double), t.R.size(), out);
        fwrite(t.Bdiv.data(), sizeof(double), t.Bdiv.size(), out);
    }
    fclose(out);
    return 0;
}
