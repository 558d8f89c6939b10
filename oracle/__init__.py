"""CPU oracle for POSLO batch verification: test infrastructure, never the product path."""
