// Host driver for the membrane element order (csrc/topology.cpp): reads
// "arity n" and n * arity node ids from stdin, prints the order.
#include <cstdio>
#include <vector>

#include "topology.h"

int main() {
    int arity = 0, n = 0;
    if (std::scanf("%d %d", &arity, &n) != 2 || arity < 1 || n < 0) return 2;
    std::vector<int> nodes((size_t)arity * n);
    for (int &v : nodes)
        if (std::scanf("%d", &v) != 1) return 2;
    const std::vector<int> order = lbib::conflict_free_order(nodes, arity, 32);
    for (int e : order) std::printf("%d\n", e);
    return 0;
}
