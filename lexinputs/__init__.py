"""Seeded input generators shared by the oracle and the GPU path.

Holds token-set specifications compiled to automata (``automaton``,
``tokensets``) and corpus generators (``corpus``).  None of the method's
arithmetic (certificates, scanning, chunk planning) lives here.
"""
