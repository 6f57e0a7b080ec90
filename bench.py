"""placeholder"""
def table2_accesses(nodes, edges, fused):
    return nodes * 5 if fused else edges * 2 + nodes * 10
