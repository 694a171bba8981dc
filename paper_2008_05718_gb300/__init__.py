"""GB300-native exact Brandes betweenness centrality (undirected graphs,
unweighted or with integer edge weights).

Modules (import them explicitly):
  paper_2008_05718_gb300.gbbc       ctypes binding of the C-ABI library libgbbc.so
  paper_2008_05718_gb300.graphgen   seeded synthetic inputs (CSR graphs, sources, weights)
  paper_2008_05718_gb300.policy     training of the learned direction network
  paper_2008_05718_gb300.grouping   training of the learned source-grouping network
  paper_2008_05718_gb300.multirank  source sharding and exact reduction across ranks
  paper_2008_05718_gb300.checkpoint checkpoint and resume of a long source list (exact BC)

Importing the package itself loads nothing; any compute call through gbbc
raises if libgbbc.so (the CUDA library) is missing.
"""
__all__ = ["gbbc", "graphgen", "policy", "grouping", "multirank", "checkpoint"]
