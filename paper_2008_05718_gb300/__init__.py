"""GB300-native exact Brandes betweenness centrality (unweighted, undirected).

Subpackages / modules (import them explicitly):
  paper_2008_05718_gb300.graphgen  seeded synthetic inputs (CSR graphs, sources)
  paper_2008_05718_gb300.gbbc      ctypes binding of the C-ABI library libgbbc.so

Importing the package itself loads nothing; any compute call through gbbc
raises if libgbbc.so (the CUDA library) is missing.
"""
__all__ = ["graphgen", "gbbc"]
