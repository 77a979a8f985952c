"""CPU oracle for the maliciously secure 3-party protocol over Z_2^64 (arXiv 2411.09287).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct restatement of the
paper's protocols on the CPU (numpy, exact integer arithmetic mod 2^l).  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``
may import it.  The product path (``paper_2411_09287_gb300``) never imports, links or calls
anything in here, and this package never imports the product.

Modules
-------
galois    Galois ring GR(2^l, d) = Z_2^l[x]/f(x) arithmetic (Sec. 2 Notation; Sec. 3).
chacha    ChaCha20 block function (RFC 8439) used as the pairwise-seeded PRG (Sec. 2).
merkle    SHA-256 Merkle hash used as H in Pi_Rec (Sec. 2, verifiable reconstruction).
shares    <.> sharings across the three simulated parties and the message ledger.
protocols Pi_<.> input sharing, Pi_Rec, Pi_Mult (Fig. MultP), Pi_Inner (Fig. DPP),
          Pi_Trunc (Fig. trunc).
verify    Pi_Tran (Fig. MTP), Pi_Reduce (Fig. Reduce), Pi_InnerVerify (Fig. DPV),
          Pi_MultVerify (Fig. PPEV), Pi_BIVerify (Fig. PBDP).

Parity status per function is stated in each module docstring.
"""
