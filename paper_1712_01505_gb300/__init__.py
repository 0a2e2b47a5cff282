"""GB300 lattice-QCD fermion solver (Kanamori & Matsufuru, arXiv:1712.01505, hot path).

The compute path is the C-ABI library ``libqcd.so`` (hand-written sm_103a CUDA);
``paper_1712_01505_gb300.qcd`` is its thin Python binding.  Importing the
package itself loads nothing, so the seeded input generators in
``paper_1712_01505_gb300.inputs`` can be used without a GPU.
"""
__all__ = ["inputs", "qcd"]
