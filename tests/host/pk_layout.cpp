// Prints pk_index (csrc/packet.h) for every (cell, entry) of a small case, one index per line,
// for tests/test_host_pk_layout.py.  Arguments: n_cell npk G.
#include <cstdio>
#include <cstdlib>

#include "packet.h"

int main(int argc, char** argv) {
    if (argc != 4) return 2;
    const long long E = atoll(argv[1]);
    const int npk = atoi(argv[2]), G = atoi(argv[3]);
    for (long long e = 0; e < E; ++e)
        for (int i = 0; i < npk; ++i) printf("%zu\n", bras::pk_index(i, e, npk, G));
    return 0;
}
